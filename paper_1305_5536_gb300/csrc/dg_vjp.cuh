// dg_vjp.cuh -- reverse-mode (vector-Jacobian) products of the 2D Euler fluxes, for
// the adjoint of the DG step: given the adjoint mu of a flux, the adjoints of the
// states it was computed from, in one reverse sweep through the flux's own
// arithmetic (instead of forward-mode dual numbers, one pass per input direction).
//
// Exact Riemann flux (Sec. 2.3; Toro's solver sampled at x/t = 0), face frame,
// primitive states (rho, u, v, p) with u normal, v transverse:
//   p* solves Phi(p) = f_L(p; rho_L, p_L) + f_R(p; rho_R, p_R) + u_R - u_L = 0,
//   u* = (u_L + u_R)/2 + (f_R(p*) - f_L(p*))/2,
//   the sampled state is side K's, its shock- or rarefaction-star state, or the
//   transonic fan, and F = (rho u, rho u^2 + p, rho u v, u (E + p)).
// The reverse sweep goes F -> sampled state -> (p*, u*, side K) -> inputs; p* by the
// implicit-function rule: an adjoint a of p* contributes -a/(f_L' + f_R') dPhi/dx.
// The derivative is that of the branch the sample lies in (the adjoint of the step
// differentiates its active branch, as for the limiter).
#pragma once

#include "dg_physics.cuh"

namespace dgk {

// Pressure function of side K (Toro's f_K) and its partial derivatives with
// respect to p, rho_K and p_K (c_K = sqrt(g p_K / rho_K) taken into account).
template <class T>
__device__ __forceinline__ void pressure_fn_partials(const Gas<T>& G, T p, T rK, T pK, T cK,
                                                     T& f, T& df, T& dr, T& dpk) {
  if (p > pK) {  // shock: f = (p - pK) sqrt(A / (p + B)), A = 2/((g+1) rho_K), B = (g-1)/(g+1) pK
    const T ipb = T(1) / (p + G.g6 * pK);
    const T q = rsqrtv(G.two_gp1 / rK * ipb);
    f = (p - pK) * q;
    df = q * (T(1) - T(0.5) * (p - pK) * ipb);
    dr = -T(0.5) * (p - pK) * q / rK;
    dpk = -q - T(0.5) * (p - pK) * q * G.g6 * ipb;
  } else {  // rarefaction: f = 2 cK/(g-1) ((p/pK)^z - 1)
    const T qz = rpow(p / pK, G.z);
    f = G.two_gm1 * cK * (qz - T(1));
    df = cK * qz * G.inv_g / p;
    dr = -T(0.5) * G.two_gm1 * (qz - T(1)) * cK / rK;
    dpk = G.two_gm1 * cK * (T(0.5) * (qz - T(1)) - G.z * qz) / pK;
  }
}

// Adjoint of the exact-solver flux: mu (mass, normal momentum, transverse momentum,
// energy) -> aL, aR, the adjoints of (rho, u, v, p) of the two sides.
template <class T>
__device__ void exact_flux_vjp(const Gas<T>& G, T rL, T uL, T vL, T pL, T rR, T uR, T vR, T pR,
                               const T* mu, T* aL, T* aR, unsigned& err) {
#pragma unroll
  for (int i = 0; i < 4; ++i) { aL[i] = T(0); aR[i] = T(0); }
  if (!(rL > T(0) && pL > T(0) && rR > T(0) && pR > T(0))) {
    err |= ERR_NONPHYS;
    return;
  }
  const T cL = rsqrtv(G.g * pL / rL), cR = rsqrtv(G.g * pR / rR);
  const T p = exact_pstar(G, rL, uL, pL, cL, rR, uR, pR, cR, err);
  T fL, dfL, fLr, fLp, fR, dfR, fRr, fRp;
  pressure_fn_partials(G, p, rL, pL, cL, fL, dfL, fLr, fLp);
  pressure_fn_partials(G, p, rR, pR, cR, fR, dfR, fRr, fRp);
  const T us = T(0.5) * (uL + uR) + T(0.5) * (fR - fL);
  // sample on the side of the contact, the right side mirrored onto the left
  const bool left = T(0) <= us;
  const T sg = left ? T(1) : T(-1);
  const T rK = left ? rL : rR, uK = left ? uL : uR, vK = left ? vL : vR;
  const T pK = left ? pL : pR, cK = left ? cL : cR;
  const T w = sg * uK, ws = sg * us, pr = p / pK;
  const bool shock = p > pK;
  bool unpert, fan = false;
  if (shock) {
    unpert = T(0) <= w - cK * rsqrtv(G.shk1 * pr + G.z);
  } else {
    unpert = T(0) <= w - cK;
    fan = !unpert && !(T(0) > ws - cK * rpow(pr, G.z));
  }
  T rho, uf, pp, c = T(0);
  if (unpert) {
    rho = rK; uf = w; pp = pK;
  } else if (shock) {
    rho = rK * (pr + G.g6) / (G.g6 * pr + T(1)); uf = ws; pp = p;
  } else if (!fan) {
    rho = rK * rpow(pr, G.inv_g); uf = ws; pp = p;
  } else {
    c = G.two_gp1 * (cK + T(0.5) * G.gm1 * w);
    uf = c;
    rho = rK * rpow(c / cK, G.two_gm1);
    pp = pK * rpow(c / cK, G.inv_z);
  }
  const T u = sg * uf;
  const T E = pp * G.inv_gm1 + T(0.5) * rho * (u * u + vK * vK);
  // F -> sampled state
  const T a_rho = mu[0] * u + mu[1] * u * u + mu[2] * u * vK + mu[3] * T(0.5) * u * (u * u + vK * vK);
  const T a_u = mu[0] * rho + T(2) * mu[1] * rho * u + mu[2] * rho * vK +
                mu[3] * ((E + pp) + rho * u * u);
  const T a_p = mu[1] + mu[3] * u * (G.inv_gm1 + T(1));
  const T a_v = mu[2] * rho * u + mu[3] * u * rho * vK;
  const T a_uf = sg * a_u;
  // sampled state -> (rho_K, u_K, p_K, c_K), p*, u*
  T a_rK = T(0), a_uK = T(0), a_pK = T(0), a_cK = T(0), a_ps = T(0), a_us = T(0);
  if (unpert) {
    a_rK = a_rho; a_uK = sg * a_uf; a_pK = a_p;
  } else if (shock) {
    const T den = G.g6 * pr + T(1);
    const T drdpr = rK * (T(1) - G.g6 * G.g6) / (den * den);
    a_rK = a_rho * (pr + G.g6) / den;
    a_ps = a_p + a_rho * drdpr / pK;
    a_pK = -a_rho * drdpr * pr / pK;
    a_us = sg * a_uf;
  } else if (!fan) {
    const T pg = rpow(pr, G.inv_g);
    const T drdpr = rK * G.inv_g * pg / pr;
    a_rK = a_rho * pg;
    a_ps = a_p + a_rho * drdpr / pK;
    a_pK = -a_rho * drdpr * pr / pK;
    a_us = sg * a_uf;
  } else {
    const T x = c / cK;
    const T xa = rpow(x, G.two_gm1), xb = rpow(x, G.inv_z);
    const T a_c = a_uf + a_rho * rK * G.two_gm1 * xa / c + a_p * pK * G.inv_z * xb / c;
    a_cK = -a_rho * rK * G.two_gm1 * xa / cK - a_p * pK * G.inv_z * xb / cK + a_c * G.two_gp1;
    a_rK = a_rho * xa;
    a_pK = a_p * xb;
    a_uK = sg * a_c * T(0.5) * G.gm1 * G.two_gp1;
  }
  // c_K = sqrt(g p_K / rho_K)
  a_rK -= a_cK * cK / (T(2) * rK);
  a_pK += a_cK * cK / (T(2) * pK);
  T* aK = left ? aL : aR;
  aK[0] += a_rK; aK[1] += a_uK; aK[2] += a_v; aK[3] += a_pK;
  // u* = (u_L + u_R)/2 + (f_R - f_L)/2
  aL[1] += T(0.5) * a_us;
  aR[1] += T(0.5) * a_us;
  a_ps += T(0.5) * a_us * (dfR - dfL);
  aL[0] -= T(0.5) * a_us * fLr;
  aL[3] -= T(0.5) * a_us * fLp;
  aR[0] += T(0.5) * a_us * fRr;
  aR[3] += T(0.5) * a_us * fRp;
  // p*: Phi(p*; x) = 0
  const T lam = a_ps / (dfL + dfR);
  aL[0] -= lam * fLr;
  aL[3] -= lam * fLp;
  aR[0] -= lam * fRr;
  aR[3] -= lam * fRp;
  aL[1] += lam;
  aR[1] -= lam;
}

// Reverse of the centroid primitives of a 2D Euler state: adjoints (a_rho, a_vx,
// a_vy, a_p) of (rho, vx, vy, p) -> adjoints of the conserved (rho, mx, my, E).
template <class T>
__device__ __forceinline__ void prims2d_vjp(const Gas<T>& G, const T* c, const T* aW, T* ac) {
  const T inv = T(1) / c[0];
  const T vx = c[1] * inv, vy = c[2] * inv;
  ac[3] = G.gm1 * aW[3];
  ac[1] = aW[1] * inv - G.gm1 * vx * aW[3];
  ac[2] = aW[2] * inv - G.gm1 * vy * aW[3];
  ac[0] = aW[0] - (aW[1] * vx + aW[2] * vy) * inv + T(0.5) * G.gm1 * (vx * vx + vy * vy) * aW[3];
}

// Adjoint of the exact flux through a face along `dir` between conserved states
// cl, cr: mu in lab-frame flux order -> the adjoints of cl and cr.
template <class T>
__device__ __forceinline__ void face_flux2d_vjp(const Gas<T>& G, int dir, const T* cl, const T* cr,
                                                const T* mu, T* acl, T* acr, unsigned& err) {
  const bool xd = dir == 0;
  const T il = T(1) / cl[0], ir = T(1) / cr[0];
  const T vxl = cl[1] * il, vyl = cl[2] * il, vxr = cr[1] * ir, vyr = cr[2] * ir;
  const T pl = G.gm1 * (cl[3] - T(0.5) * (cl[1] * vxl + cl[2] * vyl));
  const T pr = G.gm1 * (cr[3] - T(0.5) * (cr[1] * vxr + cr[2] * vyr));
  const T muf[4] = {mu[0], xd ? mu[1] : mu[2], xd ? mu[2] : mu[1], mu[3]};
  T aL[4], aR[4];
  exact_flux_vjp<T>(G, cl[0], xd ? vxl : vyl, xd ? vyl : vxl, pl, cr[0], xd ? vxr : vyr,
                    xd ? vyr : vxr, pr, muf, aL, aR, err);
  // face frame (rho, u_n, u_t, p) -> lab (rho, vx, vy, p)
  const T wl[4] = {aL[0], xd ? aL[1] : aL[2], xd ? aL[2] : aL[1], aL[3]};
  const T wr[4] = {aR[0], xd ? aR[1] : aR[2], xd ? aR[2] : aR[1], aR[3]};
  prims2d_vjp<T>(G, cl, wl, acl);
  prims2d_vjp<T>(G, cr, wr, acr);
}

// Adjoint of the physical fluxes (Fx, Fy) of a 2D Euler state c at a volume
// Gauss point: yx, yy the adjoints of Fx, Fy -> a, the adjoint of c.
template <class T>
__device__ __forceinline__ void phys_flux2d_vjp(const Gas<T>& G, const T* c, const T* yx,
                                                const T* yy, T* a) {
  const T inv = T(1) / c[0];
  const T u = c[1] * inv, v = c[2] * inv;
  const T p = G.gm1 * (c[3] - T(0.5) * (c[1] * u + c[2] * v));
  const T e = c[3] + p;
  // Fx = (mx, mx u + p, my u, e u), Fy = (my, mx v, my v + p, e v), e = E + p
  T a1 = yx[0] + yx[1] * u + yy[1] * v;
  T a2 = yy[0] + yx[2] * u + yy[2] * v;
  T au = yx[1] * c[1] + yx[2] * c[2] + yx[3] * e;
  T av = yy[1] * c[1] + yy[2] * c[2] + yy[3] * e;
  const T ae = yx[3] * u + yy[3] * v;
  const T ap = yx[1] + yy[2] + ae;
  T a3 = ae + G.gm1 * ap;
  // p = (g - 1)(E - (mx u + my v)/2)
  a1 -= T(0.5) * G.gm1 * u * ap;
  a2 -= T(0.5) * G.gm1 * v * ap;
  au -= T(0.5) * G.gm1 * c[1] * ap;
  av -= T(0.5) * G.gm1 * c[2] * ap;
  // u = mx / rho, v = my / rho
  a[1] = a1 + au * inv;
  a[2] = a2 + av * inv;
  a[0] = -(au * u + av * v) * inv;
  a[3] = a3;
}

}  // namespace dgk
