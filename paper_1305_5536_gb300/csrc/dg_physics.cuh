// dg_physics.cuh -- device physics of the P1 DG step (sm_103a).
//
// Inline device functions, templated on the arithmetic type T (double for the
// FP64 path, float for the FP32 path):
//   * gas constants and the fast magnetosonic speed (Sec. 2.1),
//   * the exact Riemann solver of the Euler equations (Sec. 2.3; Newton iteration
//     on the pressure function with the adaptive PVRS/TRRS/TSRS first guess of
//     Toro's textbook, sampled at x/t = 0),
//   * the HLLD solver of Miyoshi & Kusano (2005) for planar ideal MHD and with two
//     transverse components for 3D MHD (Sec. 2.3),
//   * the min/max slope limiter of one cell on primitive variables (Sec. 2.5).
// Face solvers work in the face frame: normal velocity u, transverse velocities,
// and return fluxes in that frame.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>

namespace dgk {

enum : unsigned {
  ERR_NONPHYS = 1u,   // rho <= 0 or p <= 0 at an evaluated state
  ERR_VACUUM = 2u,    // the exact solver met a vacuum-generating pair
  ERR_NEWTON = 4u,    // Newton iteration for p* did not converge
  ERR_TIMEOUT = 8u,   // a bounded device wait (grid barrier, TMA completion) ran out
};

template <class T> struct Prec;
template <> struct Prec<double> {
  static constexpr double newton_tol = 1e-12;
  static constexpr int newton_max = 50;
  static constexpr double hlld_degenerate = 1e-8;
};
template <> struct Prec<float> {
  static constexpr float newton_tol = 1e-5f;
  static constexpr int newton_max = 20;
  static constexpr float hlld_degenerate = 1e-8f;
};

// Powers in the exact solver (positive bases only).  FP64: the accurate pow.
// FP32: the __powf intrinsic (exp2 of e * log2 x on the special-function unit),
// a few ulp for the exponents used here, ~10x fewer instructions than powf.
__device__ __forceinline__ double rpow(double x, double e) { return pow(x, e); }
__device__ __forceinline__ float rpow(float x, float e) { return __powf(x, e); }
__device__ __forceinline__ double rsqrtv(double x) { return sqrt(x); }
__device__ __forceinline__ float rsqrtv(float x) { return sqrtf(x); }

// Conversions between the FP64 cell averages and the arithmetic type.  For the
// FP32 path they are done with integer operations on the IEEE-754 bit patterns,
// because GB300 executes FP64<->FP32 conversions on its narrow FP64 pipe.  The
// word-level rules are plain functions of the bit patterns (host and device), so
// that they can be checked on the CPU:
//   f32_bits_of_f64(hi, lo): rebias the exponent (1023 -> 127), keep the top 23
//     mantissa bits rounded to nearest (ties away from zero).  Magnitudes below
//     the smallest normal float become a zero of the same sign; magnitudes that
//     round to 2^128 or above become an infinity of the same sign; infinities stay
//     infinities and every NaN becomes the quiet NaN 0x7fc00000 (with its sign).
//   f64_words_of_f32(u): exact widening; subnormal floats become a zero of the
//     same sign, infinities and NaNs keep their class (a NaN keeps its payload).
__host__ __device__ __forceinline__ unsigned f32_bits_of_f64(unsigned h0, unsigned l0) {
  const unsigned mag = h0 & 0x7fffffffu;                   // magnitude before rounding
  const unsigned lo = l0 + 0x10000000u;                     // round at the float's last bit
  const unsigned hi = mag + (lo < l0 ? 1u : 0u);            // magnitude, with the carry
  unsigned r = ((hi - (896u << 20)) << 3) | (lo >> 29);
  r = hi < (897u << 20) ? 0u : r;                           // below the float range: zero
  r = hi >= (1151u << 20) ? 0x7f800000u : r;                // rounds to 2^128 or above: inf
  const bool special = mag >= 0x7ff00000u;                  // the double is inf or NaN
  const bool nan = mag > 0x7ff00000u || (mag == 0x7ff00000u && l0 != 0u);
  r = special ? (nan ? 0x7fc00000u : 0x7f800000u) : r;
  return r | (h0 & 0x80000000u);
}
__host__ __device__ __forceinline__ void f64_words_of_f32(unsigned u, unsigned& hi,
                                                          unsigned& lo) {
  const unsigned m = u & 0x7fffffffu;
  const unsigned e = m >= 0x7f800000u ? (0x7ff00000u | ((m & 0x007fffffu) >> 3))  // inf / NaN
                                      : ((m >> 3) + (896u << 20));
  const bool tiny = m < 0x00800000u;
  hi = (u & 0x80000000u) | (tiny ? 0u : e);
  lo = tiny ? 0u : m << 29;
}

template <class T> struct Cvt;
template <> struct Cvt<double> {
  __device__ __forceinline__ static double to_tc(double x) { return x; }
  __device__ __forceinline__ static double to_f64(double x) { return x; }
};
template <> struct Cvt<float> {
  // On the two 32-bit halves: masking the sign of the 64-bit pattern would be
  // compiled as a double absolute value, an FP64-pipe instruction.
  __device__ __forceinline__ static float to_tc(double x) {
    return __int_as_float((int)f32_bits_of_f64((unsigned)__double2hiint(x),
                                               (unsigned)__double2loint(x)));
  }
  __device__ __forceinline__ static double to_f64(float f) {
    unsigned hi, lo;
    f64_words_of_f32((unsigned)__float_as_int(f), hi, lo);
    return __hiloint2double((int)hi, (int)lo);
  }
};

// A Courant signal speed sp of a cell with density rho and pressure p that a time
// step can be taken from: finite and non-negative, and the state itself finite
// (an infinite density has zero velocity and sound speed, so sp alone would pass).
template <class T>
__device__ __forceinline__ bool courant_ok(T sp, T rho, T p) {
  const T inf = T(INFINITY);
  return sp >= T(0) && sp < inf && rho < inf && p < inf;
}

// x / 2 without the FP64 pipe: the exponent field lowered by one (integer work on
// the high word).  Exact for finite |x| >= 2^-1021; infinities and NaNs are
// returned as they are; smaller magnitudes (including zero) give a zero of the
// sign of x.
__device__ __forceinline__ double half_f64(double x) {
  const int h = __double2hiint(x), l = __double2loint(x);
  const int e = h & 0x7ff00000;
  const bool keep = e == 0x7ff00000, big = e > 0x00100000 && !keep;
  return __hiloint2double(keep ? h : (big ? h - 0x00100000 : (h & (int)0x80000000)),
                          keep || big ? l : 0);
}

// Constants of the equation of state p_gas = (gamma - 1) rho u.
template <class T>
struct Gas {
  T g, gm1, gp1, inv_gm1;
  T z;        // (g-1)/(2g)
  T inv_z;    // 2g/(g-1)
  T mzp;      // -(g+1)/(2g)
  T g6;       // (g-1)/(g+1)
  T shk1;     // (g+1)/(2g)
  T inv_g;    // 1/g
  T two_gm1;  // 2/(g-1)
  T two_gp1;  // 2/(g+1)
  __host__ __device__ void set(double gamma) {
    g = T(gamma);
    gm1 = T(gamma - 1.0);
    gp1 = T(gamma + 1.0);
    inv_gm1 = T(1.0 / (gamma - 1.0));
    z = T((gamma - 1.0) / (2.0 * gamma));
    inv_z = T(2.0 * gamma / (gamma - 1.0));
    mzp = T(-(gamma + 1.0) / (2.0 * gamma));
    g6 = T((gamma - 1.0) / (gamma + 1.0));
    shk1 = T((gamma + 1.0) / (2.0 * gamma));
    inv_g = T(1.0 / gamma);
    two_gm1 = T(2.0 / (gamma - 1.0));
    two_gp1 = T(2.0 / (gamma + 1.0));
  }
};

// Fast magnetosonic speed along a direction with normal field bn.
template <class T>
__device__ __forceinline__ T fast_speed(const Gas<T>& G, T rho, T p, T b2, T bn) {
  T a2 = G.g * p / rho;
  T bb = b2 / rho;
  T bn2 = bn * bn / rho;
  T s = a2 + bb;
  T disc = s * s - T(4) * a2 * bn2;
  disc = disc < T(0) ? T(0) : disc;
  return rsqrtv(T(0.5) * (s + rsqrtv(disc)));
}

// ----------------------------------------------------------------------------
// Exact Riemann solver (Euler).  NT transverse velocity components.
// Output F[0] mass, F[1] normal momentum, F[2..1+NT] transverse momenta,
// F[2+NT] energy -- all in the face frame.
// ----------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void pressure_fn(const Gas<T>& G, T p, T rK, T pK, T cK, T& f,
                                            T& df) {
  if (p > pK) {
    T A = G.two_gp1 / rK;
    T B = G.g6 * pK;
    T q = rsqrtv(A / (p + B));
    f = (p - pK) * q;
    df = q * (T(1) - T(0.5) * (p - pK) / (B + p));
  } else {
    // (p/pK)^(-(g+1)/(2g)) = (p/pK)^((g-1)/(2g)) / (p/pK): one power, not two
    T pr = p / pK;
    T q = rpow(pr, G.z);
    f = T(2) * cK * G.inv_gm1 * (q - T(1));
    df = q / (rK * cK * pr);
  }
}

// Star-region pressure p* of the Riemann problem (rho, u, p)_L | (rho, u, p)_R:
// root of f_L(p) + f_R(p) + (u_R - u_L) by Newton iteration from the adaptive
// PVRS / two-rarefaction / two-shock first guess.  cL, cR are the sound speeds.
template <class T>
__device__ __forceinline__ T exact_pstar(const Gas<T>& G, T rL, T uL, T pL, T cL, T rR, T uR, T pR,
                                         T cR, unsigned& err) {
  const T du = uR - uL;
  if (G.two_gm1 * (cL + cR) <= du) err |= ERR_VACUUM;
  T pv = T(0.5) * (pL + pR) - T(0.125) * du * (rL + rR) * (cL + cR);
  pv = pv > T(0) ? pv : T(0);
  const T pmin = pL < pR ? pL : pR, pmax = pL < pR ? pR : pL;
  T p;
  if (pmax / pmin <= T(2) && pmin <= pv && pv <= pmax) {
    p = pv;
  } else if (pv < pmin) {
    T num = cL + cR - T(0.5) * G.gm1 * du;
    T den = cL / rpow(pL, G.z) + cR / rpow(pR, G.z);
    p = rpow((num > T(0) ? num : T(0)) / den, G.inv_z);
  } else {
    T gL = rsqrtv(G.two_gp1 / rL / (G.g6 * pL + pv));
    T gR = rsqrtv(G.two_gp1 / rR / (G.g6 * pR + pv));
    p = (gL * pL + gR * pR - du) / (gL + gR);
  }
  const T pfloor = T(1e-10) * pmin;
  if (!(p > pfloor)) p = pfloor;
  bool conv = false;
  for (int it = 0; it < Prec<T>::newton_max; ++it) {
    T fL, dfL, fR, dfR;
    pressure_fn(G, p, rL, pL, cL, fL, dfL);
    pressure_fn(G, p, rR, pR, cR, fR, dfR);
    T pn = p - (fL + fR + du) / (dfL + dfR);
    if (!(pn > pfloor)) pn = pfloor;
    T change = T(2) * fabs(pn - p) / (pn + p);
    p = pn;
    if (change < Prec<T>::newton_tol) { conv = true; break; }
  }
  if (!conv) err |= ERR_NEWTON;
  return p;
}

template <int NT>
__device__ __forceinline__ void exact_flux_f32(const Gas<float>& G, float rL, float uL, float pL,
                                               const float* vtL, float rR, float uR, float pR,
                                               const float* vtR, float* F, unsigned& err);

template <class T, int NT>
__device__ __forceinline__ void exact_flux(const Gas<T>& G, T rL, T uL, T pL, const T* vtL, T rR,
                                           T uR, T pR, const T* vtR, T* F, unsigned& err) {
  if constexpr (std::is_same<T, float>::value) {
    exact_flux_f32<NT>(G, rL, uL, pL, vtL, rR, uR, pR, vtR, F, err);
    return;
  }
  if (!(rL > T(0) && pL > T(0) && rR > T(0) && pR > T(0))) {
    err |= ERR_NONPHYS;
    for (int q = 0; q < 3 + NT; ++q) F[q] = T(0);
    return;
  }
  const T cL = rsqrtv(G.g * pL / rL), cR = rsqrtv(G.g * pR / rR);
  const T p = exact_pstar(G, rL, uL, pL, cL, rR, uR, pR, cR, err);
  T fL, dfL, fR, dfR;
  pressure_fn(G, p, rL, pL, cL, fL, dfL);
  pressure_fn(G, p, rR, pR, cR, fR, dfR);
  const T us = T(0.5) * (uL + uR) + T(0.5) * (fR - fL);
  // sample the self-similar solution at x/t = 0
  T rho, u, pp;
  const T* vt;
  if (T(0) <= us) {
    vt = vtL;
    if (p > pL) {
      T SL = uL - cL * rsqrtv(G.shk1 * p / pL + G.z);
      if (T(0) <= SL) { rho = rL; u = uL; pp = pL; }
      else { rho = rL * ((p / pL + G.g6) / (G.g6 * p / pL + T(1))); u = us; pp = p; }
    } else {
      T SHL = uL - cL;
      if (T(0) <= SHL) { rho = rL; u = uL; pp = pL; }
      else {
        T cmL = cL * rpow(p / pL, G.z);
        if (T(0) > us - cmL) { rho = rL * rpow(p / pL, G.inv_g); u = us; pp = p; }
        else {
          T c = G.two_gp1 * (cL + T(0.5) * G.gm1 * uL);
          u = c;
          rho = rL * rpow(c / cL, G.two_gm1);
          pp = pL * rpow(c / cL, G.inv_z);
        }
      }
    }
  } else {
    vt = vtR;
    if (p > pR) {
      T SR = uR + cR * rsqrtv(G.shk1 * p / pR + G.z);
      if (T(0) >= SR) { rho = rR; u = uR; pp = pR; }
      else { rho = rR * ((p / pR + G.g6) / (G.g6 * p / pR + T(1))); u = us; pp = p; }
    } else {
      T SHR = uR + cR;
      if (T(0) >= SHR) { rho = rR; u = uR; pp = pR; }
      else {
        T cmR = cR * rpow(p / pR, G.z);
        if (T(0) < us + cmR) { rho = rR * rpow(p / pR, G.inv_g); u = us; pp = p; }
        else {
          T c = G.two_gp1 * (cR - T(0.5) * G.gm1 * uR);
          u = -c;
          rho = rR * rpow(c / cR, G.two_gm1);
          pp = pR * rpow(c / cR, G.inv_z);
        }
      }
    }
  }
  T kin = u * u;
#pragma unroll
  for (int a = 0; a < NT; ++a) kin += vt[a] * vt[a];
  const T E = pp * G.inv_gm1 + T(0.5) * rho * kin;
  const T mu = rho * u;
  F[0] = mu;
  F[1] = mu * u + pp;
#pragma unroll
  for (int a = 0; a < NT; ++a) F[2 + a] = mu * vt[a];
  F[2 + NT] = u * (E + pp);
}

// ----------------------------------------------------------------------------
// The exact Riemann solver of the FP32 path.  It computes the solution of
// exact_flux (Toro's exact solver: Newton iteration for p* on f_L + f_R + du = 0
// from the adaptive PVRS / TRRS / TSRS guess, sampled at x/t = 0) with the
// arithmetic arranged for the FP32 pipes:
//   * per side, the constants of the pressure function are formed once:
//       shock       f = (p - pK) q,  q = (A_K / (p + B_K))^(1/2),
//                   f' = q (1 - (p - pK) / (2 (p + B_K))) = q (1 - (p - pK) q^2 / (2 A_K)),
//       rarefaction f = 2 cK / (g - 1) ((p/pK)^z - 1),  f' = (p/pK)^z cK / (g p),
//     with A_K = 2 / ((g + 1) rho_K), B_K = (g - 1) / (g + 1) pK, z = (g - 1) / (2g);
//     divisions become approximate reciprocals, square roots reciprocal square
//     roots, powers exp2(e log2 x) (all within a few ulp);
//   * both branches of f are evaluated and one is selected, so that lanes of a
//     warp on different branches (near-equal states put p on either side of pK
//     at random) do not serialise;
//   * Newton converges quadratically: accepting the update p_n after a step of
//     relative size delta leaves an error of about k delta^2 (k <= 1/2 for these
//     pressure functions), so steps below 2e-4 are accepted (error < 2e-8, below
//     the FP32 evaluation noise of f), and f_K(p*) for u* is taken from the last
//     iteration's linearisation f_K(p) + f_K'(p)(p* - p) (error O(delta^2) again);
//   * the sampling picks the side of the contact by select and mirrors the right
//     side onto the left (u -> -u), so the unperturbed / shock-star /
//     rarefaction-star choice is a select; only the transonic rarefaction fan,
//     which is rare, is a branch.
// ----------------------------------------------------------------------------
__device__ __forceinline__ float rcpf(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ float sqrtf_pos(float x) { return x * rsqrtf(x); }  // x > 0

template <int NT>
__device__ __forceinline__ void exact_flux_f32(const Gas<float>& G, float rL, float uL, float pL,
                                               const float* vtL, float rR, float uR, float pR,
                                               const float* vtR, float* F, unsigned& err) {
  if (!(rL > 0.0f && pL > 0.0f && rR > 0.0f && pR > 0.0f)) {
    err |= ERR_NONPHYS;
    for (int q = 0; q < 3 + NT; ++q) F[q] = 0.0f;
    return;
  }
  constexpr float accept = 2e-4f;
  const float ipL = rcpf(pL), ipR = rcpf(pR);
  const float aL = G.g * pL * rcpf(rL), aR = G.g * pR * rcpf(rR);
  const float cL = sqrtf_pos(aL), cR = sqrtf_pos(aR);
  const float AiL = 0.5f * G.gp1 * rL, AiR = 0.5f * G.gp1 * rR;  // 1 / A_K
  const float BL = G.g6 * pL, BR = G.g6 * pR;
  const float CL = G.two_gm1 * cL, CR = G.two_gm1 * cR;          // 2 cK / (g - 1)
  const float DL = cL * G.inv_g, DR = cR * G.inv_g;              // cK / g
  const float du = uR - uL;
  if (CL + CR <= du) err |= ERR_VACUUM;
  // first guess (Toro's adaptive choice)
  const float pmin = fminf(pL, pR), pmax = fmaxf(pL, pR);
  float pv = 0.5f * (pL + pR) - 0.125f * du * (rL + rR) * (cL + cR);
  pv = fmaxf(pv, 0.0f);
  float p = pv;
  if (!(pmax <= 2.0f * pmin && pmin <= pv && pv <= pmax)) {
    if (pv < pmin) {  // two rarefactions
      const float num = fmaxf(cL + cR - 0.5f * G.gm1 * du, 0.0f);
      const float den = cL * exp2f(-G.z * __log2f(pL)) + cR * exp2f(-G.z * __log2f(pR));
      p = exp2f(G.inv_z * __log2f(num * rcpf(den)));
    } else {  // two shocks
      const float gL = rsqrtf((BL + pv) * AiL), gR = rsqrtf((BR + pv) * AiR);
      p = (gL * pL + gR * pR - du) * rcpf(gL + gR);
    }
  }
  const float pfloor = 1e-10f * pmin;
  if (!(p > pfloor)) p = pfloor;
  // Newton iteration; fL, fR, dfL, dfR, p0 keep the last linearisation
  float fL = 0.0f, fR = 0.0f, dfL = 1.0f, dfR = 1.0f, p0 = p;
  bool conv = false;
  for (int it = 0; it < Prec<float>::newton_max; ++it) {
    const float rp = rcpf(p);
    {
      const float dp = p - pL;
      const float q = rsqrtf((p + BL) * AiL);
      const float fs = dp * q, dfs = q * (1.0f - 0.5f * dp * q * q * AiL);
      const float qr = exp2f(G.z * __log2f(p * ipL));
      const float fr = CL * (qr - 1.0f), dfr = qr * DL * rp;
      const bool sh = p > pL;
      fL = sh ? fs : fr;
      dfL = sh ? dfs : dfr;
    }
    {
      const float dp = p - pR;
      const float q = rsqrtf((p + BR) * AiR);
      const float fs = dp * q, dfs = q * (1.0f - 0.5f * dp * q * q * AiR);
      const float qr = exp2f(G.z * __log2f(p * ipR));
      const float fr = CR * (qr - 1.0f), dfr = qr * DR * rp;
      const bool sh = p > pR;
      fR = sh ? fs : fr;
      dfR = sh ? dfs : dfr;
    }
    float pn = p - (fL + fR + du) * rcpf(dfL + dfR);
    if (!(pn > pfloor)) pn = pfloor;
    p0 = p;
    const bool done = 2.0f * fabsf(pn - p) < accept * (pn + p);
    p = pn;
    if (done) { conv = true; break; }
  }
  if (!conv) err |= ERR_NEWTON;
  // u* from the pressure functions at p*, by the last linearisation
  const float dps = p - p0;
  const float us = 0.5f * (uL + uR) + 0.5f * ((fR + dfR * dps) - (fL + dfL * dps));
  // sample at x/t = 0 on the side of the contact that x/t = 0 lies on, the right
  // side mirrored onto the left (velocities negated)
  const bool left = us >= 0.0f;
  const float sg = left ? 1.0f : -1.0f;
  const float rK = left ? rL : rR, pK = left ? pL : pR, cK = left ? cL : cR;
  const float ipK = left ? ipL : ipR;
  const float w = sg * (left ? uL : uR), ws = sg * us;
  const float pr = p * ipK;
  const bool shock = p > pK;
  const float Ssh = w - cK * sqrtf_pos(G.shk1 * pr + G.z);         // shock speed
  const float rsh = rK * (pr + G.g6) * rcpf(G.g6 * pr + 1.0f);      // behind the shock
  const float lpr = __log2f(pr);
  const float cm = cK * exp2f(G.z * lpr);                           // sound speed behind the fan
  const float rrf = rK * exp2f(G.inv_g * lpr);                      // isentropic star density
  const bool unpert = shock ? Ssh >= 0.0f : w - cK >= 0.0f;
  const bool fan = !shock && !unpert && !(ws - cm < 0.0f);
  float rho = unpert ? rK : (shock ? rsh : rrf);
  float u = unpert ? w : ws;
  float pp = unpert ? pK : p;
  if (fan) {
    const float c = G.two_gp1 * (cK + 0.5f * G.gm1 * w);
    const float lc = __log2f(c * rcpf(cK));
    u = c;
    rho = rK * exp2f(G.two_gm1 * lc);
    pp = pK * exp2f(G.inv_z * lc);
  }
  u *= sg;
  float vt[NT > 0 ? NT : 1];
  float kin = u * u;
#pragma unroll
  for (int a = 0; a < NT; ++a) {
    vt[a] = left ? vtL[a] : vtR[a];
    kin += vt[a] * vt[a];
  }
  const float E = pp * G.inv_gm1 + 0.5f * rho * kin;
  const float mu = rho * u;
  F[0] = mu;
  F[1] = mu * u + pp;
#pragma unroll
  for (int a = 0; a < NT; ++a) F[2 + a] = mu * vt[a];
  F[2 + NT] = u * (E + pp);
}

// ----------------------------------------------------------------------------
// HLLD solver, planar MHD (one transverse velocity v and field bt; out-of-plane
// components are zero).  bn is the common normal field.  Output in the face
// frame: F[0] mass, F[1] normal momentum, F[2] transverse momentum, F[3] energy,
// F[4] flux of the transverse field (the normal-field flux is zero).
// ----------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void hlld_flux(const Gas<T>& G, T rL, T uL, T vL, T pL, T btL, T rR,
                                          T uR, T vR, T pR, T btR, T bn, T* F, unsigned& err) {
  if (!(rL > T(0) && pL > T(0) && rR > T(0) && pR > T(0))) {
    err |= ERR_NONPHYS;
    for (int q = 0; q < 5; ++q) F[q] = T(0);
    return;
  }
  const T bn2 = bn * bn;
  const T b2L = bn2 + btL * btL, b2R = bn2 + btR * btR;
  const T EL = pL * G.inv_gm1 + T(0.5) * rL * (uL * uL + vL * vL) + T(0.5) * b2L;
  const T ER = pR * G.inv_gm1 + T(0.5) * rR * (uR * uR + vR * vR) + T(0.5) * b2R;
  const T pTL = pL + T(0.5) * b2L, pTR = pR + T(0.5) * b2R;
  const T cfL = fast_speed(G, rL, pL, b2L, bn), cfR = fast_speed(G, rR, pR, b2R, bn);
  const T cmax = cfL > cfR ? cfL : cfR;
  const T SL = (uL < uR ? uL : uR) - cmax;
  const T SR = (uL < uR ? uR : uL) + cmax;
  // physical fluxes and conserved vectors of both sides
  T FL[5], FR[5], UL[5], UR[5];
  {
    T vB = uL * bn + vL * btL;
    FL[0] = rL * uL; FL[1] = rL * uL * uL + pTL - bn2; FL[2] = rL * uL * vL - bn * btL;
    FL[3] = (EL + pTL) * uL - bn * vB; FL[4] = btL * uL - vL * bn;
    UL[0] = rL; UL[1] = rL * uL; UL[2] = rL * vL; UL[3] = EL; UL[4] = btL;
    vB = uR * bn + vR * btR;
    FR[0] = rR * uR; FR[1] = rR * uR * uR + pTR - bn2; FR[2] = rR * uR * vR - bn * btR;
    FR[3] = (ER + pTR) * uR - bn * vB; FR[4] = btR * uR - vR * bn;
    UR[0] = rR; UR[1] = rR * uR; UR[2] = rR * vR; UR[3] = ER; UR[4] = btR;
  }
  if (SL > T(0)) {
    for (int q = 0; q < 5; ++q) F[q] = FL[q];
    return;
  }
  if (SR < T(0)) {
    for (int q = 0; q < 5; ++q) F[q] = FR[q];
    return;
  }
  const T dL = SL - uL, dR = SR - uR;
  const T den = dR * rR - dL * rL;
  const T SM = (dR * rR * uR - dL * rL * uL - pTR + pTL) / den;
  const T pTs = (dR * rR * pTL - dL * rL * pTR + rL * rR * dR * dL * (uR - uL)) / den;
  // single-star states
  T rsL, vsL, btsL, EsL, rsR, vsR, btsR, EsR;
  {
    T dd = rL * dL * (SL - SM) - bn2;
    rsL = rL * dL / (SL - SM);
    if (fabs(dd) < Prec<T>::hlld_degenerate * (rL * dL * dL + bn2)) {
      vsL = vL; btsL = btL;
    } else {
      T tv = bn * (SM - uL) / dd;
      T tb = (rL * dL * dL - bn2) / dd;
      vsL = vL - btL * tv;
      btsL = btL * tb;
    }
    T vB = uL * bn + vL * btL, vBs = SM * bn + vsL * btsL;
    EsL = (dL * EL - pTL * uL + pTs * SM + bn * (vB - vBs)) / (SL - SM);
    dd = rR * dR * (SR - SM) - bn2;
    rsR = rR * dR / (SR - SM);
    if (fabs(dd) < Prec<T>::hlld_degenerate * (rR * dR * dR + bn2)) {
      vsR = vR; btsR = btR;
    } else {
      T tv = bn * (SM - uR) / dd;
      T tb = (rR * dR * dR - bn2) / dd;
      vsR = vR - btR * tv;
      btsR = btR * tb;
    }
    vB = uR * bn + vR * btR;
    vBs = SM * bn + vsR * btsR;
    EsR = (dR * ER - pTR * uR + pTs * SM + bn * (vB - vBs)) / (SR - SM);
  }
  T UsL[5] = {rsL, rsL * SM, rsL * vsL, EsL, btsL};
  T UsR[5] = {rsR, rsR * SM, rsR * vsR, EsR, btsR};
  const T sqL = rsqrtv(rsL), sqR = rsqrtv(rsR);
  const T SsL = SM - fabs(bn) / sqL, SsR = SM + fabs(bn) / sqR;
  if (SsL >= T(0)) {
    for (int q = 0; q < 5; ++q) F[q] = FL[q] + SL * (UsL[q] - UL[q]);
    return;
  }
  if (SsR <= T(0)) {
    for (int q = 0; q < 5; ++q) F[q] = FR[q] + SR * (UsR[q] - UR[q]);
    return;
  }
  // double-star states between the Alfven waves
  const T sg = bn > T(0) ? T(1) : (bn < T(0) ? T(-1) : T(0));
  const T inv = T(1) / (sqL + sqR);
  const T vss = (sqL * vsL + sqR * vsR + (btsR - btsL) * sg) * inv;
  const T btss = (sqL * btsR + sqR * btsL + sqL * sqR * (vsR - vsL) * sg) * inv;
  const T vBss = SM * bn + vss * btss;
  if (SM >= T(0)) {
    T vBsL = SM * bn + vsL * btsL;
    T E2 = EsL - sqL * (vBsL - vBss) * sg;
    T U2[5] = {rsL, rsL * SM, rsL * vss, E2, btss};
    for (int q = 0; q < 5; ++q)
      F[q] = FL[q] + SL * (UsL[q] - UL[q]) + SsL * (U2[q] - UsL[q]);
  } else {
    T vBsR = SM * bn + vsR * btsR;
    T E2 = EsR + sqR * (vBsR - vBss) * sg;
    T U2[5] = {rsR, rsR * SM, rsR * vss, E2, btss};
    for (int q = 0; q < 5; ++q)
      F[q] = FR[q] + SR * (UsR[q] - UR[q]) + SsR * (U2[q] - UsR[q]);
  }
}

// ----------------------------------------------------------------------------
// HLLD solver with two transverse components (3D MHD): per side (rho, u, v, w, p,
// bv, bw) with u normal and (v, w), (bv, bw) the transverse velocity and field;
// bn the common normal field.  Output in the face frame: F[0] mass, F[1] normal
// momentum, F[2], F[3] transverse momenta, F[4] energy, F[5], F[6] transverse
// field fluxes (the normal-field flux is zero).  Same wave-speed estimates and
// degeneracy switch as hlld_flux.
// ----------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void hlld_flux3(const Gas<T>& G, T rL, T uL, T vL, T wL, T pL, T bvL,
                                           T bwL, T rR, T uR, T vR, T wR, T pR, T bvR, T bwR,
                                           T bn, T* F, unsigned& err) {
  if (!(rL > T(0) && pL > T(0) && rR > T(0) && pR > T(0))) {
    err |= ERR_NONPHYS;
    for (int q = 0; q < 7; ++q) F[q] = T(0);
    return;
  }
  const T bn2 = bn * bn;
  const T b2L = bn2 + bvL * bvL + bwL * bwL, b2R = bn2 + bvR * bvR + bwR * bwR;
  const T EL = pL * G.inv_gm1 + T(0.5) * rL * (uL * uL + vL * vL + wL * wL) + T(0.5) * b2L;
  const T ER = pR * G.inv_gm1 + T(0.5) * rR * (uR * uR + vR * vR + wR * wR) + T(0.5) * b2R;
  const T pTL = pL + T(0.5) * b2L, pTR = pR + T(0.5) * b2R;
  const T cfL = fast_speed(G, rL, pL, b2L, bn), cfR = fast_speed(G, rR, pR, b2R, bn);
  const T cmax = cfL > cfR ? cfL : cfR;
  const T SL = (uL < uR ? uL : uR) - cmax;
  const T SR = (uL < uR ? uR : uL) + cmax;
  T FL[7], FR[7], UL[7], UR[7];
  {
    T vB = uL * bn + vL * bvL + wL * bwL;
    FL[0] = rL * uL; FL[1] = rL * uL * uL + pTL - bn2; FL[2] = rL * uL * vL - bn * bvL;
    FL[3] = rL * uL * wL - bn * bwL; FL[4] = (EL + pTL) * uL - bn * vB;
    FL[5] = bvL * uL - vL * bn; FL[6] = bwL * uL - wL * bn;
    UL[0] = rL; UL[1] = rL * uL; UL[2] = rL * vL; UL[3] = rL * wL; UL[4] = EL;
    UL[5] = bvL; UL[6] = bwL;
    vB = uR * bn + vR * bvR + wR * bwR;
    FR[0] = rR * uR; FR[1] = rR * uR * uR + pTR - bn2; FR[2] = rR * uR * vR - bn * bvR;
    FR[3] = rR * uR * wR - bn * bwR; FR[4] = (ER + pTR) * uR - bn * vB;
    FR[5] = bvR * uR - vR * bn; FR[6] = bwR * uR - wR * bn;
    UR[0] = rR; UR[1] = rR * uR; UR[2] = rR * vR; UR[3] = rR * wR; UR[4] = ER;
    UR[5] = bvR; UR[6] = bwR;
  }
  if (SL > T(0)) {
    for (int q = 0; q < 7; ++q) F[q] = FL[q];
    return;
  }
  if (SR < T(0)) {
    for (int q = 0; q < 7; ++q) F[q] = FR[q];
    return;
  }
  const T dL = SL - uL, dR = SR - uR;
  const T den = dR * rR - dL * rL;
  const T SM = (dR * rR * uR - dL * rL * uL - pTR + pTL) / den;
  const T pTs = (dR * rR * pTL - dL * rL * pTR + rL * rR * dR * dL * (uR - uL)) / den;
  // single-star states
  T rsL, vsL, wsL, bvsL, bwsL, EsL, rsR, vsR, wsR, bvsR, bwsR, EsR;
  {
    T dd = rL * dL * (SL - SM) - bn2;
    rsL = rL * dL / (SL - SM);
    if (fabs(dd) < Prec<T>::hlld_degenerate * (rL * dL * dL + bn2)) {
      vsL = vL; wsL = wL; bvsL = bvL; bwsL = bwL;
    } else {
      T tv = bn * (SM - uL) / dd;
      T tb = (rL * dL * dL - bn2) / dd;
      vsL = vL - bvL * tv; wsL = wL - bwL * tv;
      bvsL = bvL * tb; bwsL = bwL * tb;
    }
    T vB = uL * bn + vL * bvL + wL * bwL, vBs = SM * bn + vsL * bvsL + wsL * bwsL;
    EsL = (dL * EL - pTL * uL + pTs * SM + bn * (vB - vBs)) / (SL - SM);
    dd = rR * dR * (SR - SM) - bn2;
    rsR = rR * dR / (SR - SM);
    if (fabs(dd) < Prec<T>::hlld_degenerate * (rR * dR * dR + bn2)) {
      vsR = vR; wsR = wR; bvsR = bvR; bwsR = bwR;
    } else {
      T tv = bn * (SM - uR) / dd;
      T tb = (rR * dR * dR - bn2) / dd;
      vsR = vR - bvR * tv; wsR = wR - bwR * tv;
      bvsR = bvR * tb; bwsR = bwR * tb;
    }
    vB = uR * bn + vR * bvR + wR * bwR;
    vBs = SM * bn + vsR * bvsR + wsR * bwsR;
    EsR = (dR * ER - pTR * uR + pTs * SM + bn * (vB - vBs)) / (SR - SM);
  }
  T UsL[7] = {rsL, rsL * SM, rsL * vsL, rsL * wsL, EsL, bvsL, bwsL};
  T UsR[7] = {rsR, rsR * SM, rsR * vsR, rsR * wsR, EsR, bvsR, bwsR};
  const T sqL = rsqrtv(rsL), sqR = rsqrtv(rsR);
  const T SsL = SM - fabs(bn) / sqL, SsR = SM + fabs(bn) / sqR;
  if (SsL >= T(0)) {
    for (int q = 0; q < 7; ++q) F[q] = FL[q] + SL * (UsL[q] - UL[q]);
    return;
  }
  if (SsR <= T(0)) {
    for (int q = 0; q < 7; ++q) F[q] = FR[q] + SR * (UsR[q] - UR[q]);
    return;
  }
  // double-star states between the Alfven waves
  const T sg = bn > T(0) ? T(1) : (bn < T(0) ? T(-1) : T(0));
  const T inv = T(1) / (sqL + sqR);
  const T vss = (sqL * vsL + sqR * vsR + (bvsR - bvsL) * sg) * inv;
  const T wss = (sqL * wsL + sqR * wsR + (bwsR - bwsL) * sg) * inv;
  const T bvss = (sqL * bvsR + sqR * bvsL + sqL * sqR * (vsR - vsL) * sg) * inv;
  const T bwss = (sqL * bwsR + sqR * bwsL + sqL * sqR * (wsR - wsL) * sg) * inv;
  const T vBss = SM * bn + vss * bvss + wss * bwss;
  if (SM >= T(0)) {
    T vBsL = SM * bn + vsL * bvsL + wsL * bwsL;
    T E2 = EsL - sqL * (vBsL - vBss) * sg;
    T U2[7] = {rsL, rsL * SM, rsL * vss, rsL * wss, E2, bvss, bwss};
    for (int q = 0; q < 7; ++q)
      F[q] = FL[q] + SL * (UsL[q] - UL[q]) + SsL * (U2[q] - UsL[q]);
  } else {
    T vBsR = SM * bn + vsR * bvsR + wsR * bwsR;
    T E2 = EsR + sqR * (vBsR - vBss) * sg;
    T U2[7] = {rsR, rsR * SM, rsR * vss, rsR * wss, E2, bvss, bwss};
    for (int q = 0; q < 7; ++q)
      F[q] = FR[q] + SR * (UsR[q] - UR[q]) + SsR * (U2[q] - UsR[q]);
  }
}

// ----------------------------------------------------------------------------
// Min/max limiter coefficient of one primitive (Sec. 2.5):
//   alpha = min(1, min_faces psi_f), psi_f = (phimax - phi)/dphi_f (dphi_f > 0),
//   (phimin - phi)/dphi_f (dphi_f < 0), 1 (dphi_f = 0), dphi_f = grad phi . (f - s).
// On a Cartesian cell the faces along axis d have dphi = +-a_d with
// a_d = g_d h_d / 2, so min_faces psi = min(phimax - phi, phi - phimin) / max_d |a_d|
// (division is monotone, so this is the same floating-point value).
// ----------------------------------------------------------------------------
template <class T, int DIM>
__device__ __forceinline__ T limiter_alpha(T phi, T phimax, T phimin, const T* grad,
                                           const T* half_h) {
  T amax = T(0);
#pragma unroll
  for (int d = 0; d < DIM; ++d) {
    T a = fabs(grad[d] * half_h[d]);
    amax = a > amax ? a : amax;
  }
  if (!(amax > T(0))) return T(1);
  T up = phimax - phi, dn = phi - phimin;
  T m = up < dn ? up : dn;
  T psi = m / amax;
  return psi < T(1) ? psi : T(1);
}

}  // namespace dgk
