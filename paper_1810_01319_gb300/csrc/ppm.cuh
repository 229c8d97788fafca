// Per-cell and per-interface arithmetic of the PPM sweep (Sec. II.C: the
// hydro Method is a modified piecewise parabolic method, Colella & Woodward
// 1984).  Every expression is written in a fixed evaluation order so that the
// float64 build (compiled without FMA contraction) rounds exactly like a
// plain float64 evaluation of the same formulas.
#pragma once

#include <cuda_runtime.h>

#include <cmath>

#ifndef CELLO_HD
#define CELLO_HD __host__ __device__ __forceinline__
#endif

namespace cello {

constexpr double kRhoFloor = 1e-10;
constexpr double kPFloor = 1e-20;
constexpr double kEpsShock = 0.33;   // shock detector: relative pressure jump
constexpr double kOmega1 = 0.75;     // flattening ratio offset
constexpr double kOmega2 = 10.0;     // flattening ratio slope
constexpr int kRiemannIters = 5;     // Newton steps (a lane stops early only at an exact fixed point)

template <typename T> CELLO_HD T vmax(T a, T b) { return a > b ? a : b; }
template <typename T> CELLO_HD T vmin(T a, T b) { return a < b ? a : b; }
CELLO_HD float vabs(float a) { return fabsf(a); }
CELLO_HD double vabs(double a) { return fabs(a); }
CELLO_HD float vsqrt(float a) { return sqrtf(a); }
CELLO_HD double vsqrt(double a) { return sqrt(a); }
CELLO_HD float vcopysign(float a, float b) { return copysignf(a, b); }
CELLO_HD double vcopysign(double a, double b) { return copysign(a, b); }

// Subtraction that is never fused with the multiply producing an operand
// (a flux difference must round each flux first, wherever the fluxes live).
CELLO_HD float sub_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}
CELLO_HD double sub_rn(double a, double b) {
#ifdef __CUDA_ARCH__
  return __dsub_rn(a, b);
#else
  return a - b;
#endif
}

// Division in the bulk arithmetic: float32 on the device uses the fast
// approximate form (reciprocal and multiply, within 2 ulp for divisors
// below 2^126, which every divisor here is: densities, pressures, sound
// speeds and their sums); float64 keeps the correctly rounded division.
CELLO_HD float vdiv(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fdividef(a, b);
#else
  return a / b;
#endif
}
CELLO_HD double vdiv(double a, double b) { return a / b; }

// Gas constants in the working precision, derived once in float64.
template <typename T> struct Gas {
  T gamma, gm1, g1, inv_gm1;
  __host__ __device__ static Gas make(double gamma) {
    Gas s;
    s.gamma = T(gamma);
    s.gm1 = T(gamma - 1.0);
    s.g1 = T((gamma + 1.0) / (2.0 * gamma));
    s.inv_gm1 = T(1.0 / (gamma - 1.0));
    return s;
  }
};

// Conserved (rho, m_n, m_t1, m_t2, E) -> primitive (rho, u_n, u_t1, u_t2, p).
template <typename T>
CELLO_HD void to_primitive(const T U[5], const Gas<T>& gs, T W[5]) {
  T rho = vmax(U[0], T(kRhoFloor));
  T un = U[1] / rho;
  T ut1 = U[2] / rho;
  T ut2 = U[3] / rho;
  T ke = (T(0.5) * rho) * (un * un + (ut1 * ut1 + ut2 * ut2));
  T p = vmax(gs.gm1 * (U[4] - ke), T(kPFloor));
  W[0] = rho; W[1] = un; W[2] = ut1; W[3] = ut2; W[4] = p;
}

// Float32 form: one reciprocal of rho and three multiplies rounded on their
// own (never fused into a neighbouring add), so that a velocity is the same
// rounded value whether it is kept in a register or passes through memory.
CELLO_HD void to_primitive(const float U[5], const Gas<float>& gs, float W[5]) {
  const float rho = vmax(U[0], float(kRhoFloor));
  const float ir = vdiv(1.0f, rho);
#ifdef __CUDA_ARCH__
  const float un = __fmul_rn(U[1], ir), ut1 = __fmul_rn(U[2], ir), ut2 = __fmul_rn(U[3], ir);
#else
  const float un = U[1] * ir, ut1 = U[2] * ir, ut2 = U[3] * ir;
#endif
  const float ke = (0.5f * rho) * (un * un + (ut1 * ut1 + ut2 * ut2));
  const float p = vmax(gs.gm1 * (U[4] - ke), float(kPFloor));
  W[0] = rho; W[1] = un; W[2] = ut1; W[3] = ut2; W[4] = p;
}

// Dual-energy formalism (Bryan et al. 1995): a sixth field, the internal
// energy density rho e.  The pressure comes from E - ke where that exceeds
// kDualEta1 E, else from rho e; after a sweep's update rho e is reset to
// E - ke where that exceeds kDualEta2 E.
constexpr double kDualEta1 = 1e-3;
constexpr double kDualEta2 = 0.1;

// (rho, m_n, m_t1, m_t2, E, rho e) -> (rho, u_n, u_t1, u_t2, p, e).
template <typename T>
CELLO_HD void to_primitive_de(const T U[6], const Gas<T>& gs, T W[6]) {
  T rho = vmax(U[0], T(kRhoFloor));
  T un = U[1] / rho;
  T ut1 = U[2] / rho;
  T ut2 = U[3] / rho;
  T ke = (T(0.5) * rho) * (un * un + (ut1 * ut1 + ut2 * ut2));
  const T eint = U[4] - ke;
  const T src = (eint > T(kDualEta1) * U[4]) ? eint : U[5];
  W[0] = rho; W[1] = un; W[2] = ut1; W[3] = ut2;
  W[4] = vmax(gs.gm1 * src, T(kPFloor));
  W[5] = U[5] / rho;
}

CELLO_HD void to_primitive_de(const float U[6], const Gas<float>& gs, float W[6]) {
  const float rho = vmax(U[0], float(kRhoFloor));
  const float ir = vdiv(1.0f, rho);
#ifdef __CUDA_ARCH__
  const float un = __fmul_rn(U[1], ir), ut1 = __fmul_rn(U[2], ir), ut2 = __fmul_rn(U[3], ir);
  const float e = __fmul_rn(U[5], ir);
#else
  const float un = U[1] * ir, ut1 = U[2] * ir, ut2 = U[3] * ir, e = U[5] * ir;
#endif
  const float ke = (0.5f * rho) * (un * un + (ut1 * ut1 + ut2 * ut2));
  const float eint = U[4] - ke;
  const float src = (eint > float(kDualEta1) * U[4]) ? eint : U[5];
  W[0] = rho; W[1] = un; W[2] = ut1; W[3] = ut2;
  W[4] = vmax(gs.gm1 * src, float(kPFloor));
  W[5] = e;
}

// The synchronised rho e of an updated cell (sweep-ordered state U[6]).
template <typename T>
CELLO_HD T dual_sync(const T U[6]) {
  T rho = vmax(U[0], T(kRhoFloor));
  T un = U[1] / rho;
  T ut1 = U[2] / rho;
  T ut2 = U[3] / rho;
  T ke = (T(0.5) * rho) * (un * un + (ut1 * ut1 + ut2 * ut2));
  const T eint = U[4] - ke;
  return (eint > T(kDualEta2) * U[4]) ? eint : U[5];
}

CELLO_HD float dual_sync(const float U[6]) {
  const float rho = vmax(U[0], float(kRhoFloor));
  const float ir = vdiv(1.0f, rho);
#ifdef __CUDA_ARCH__
  const float un = __fmul_rn(U[1], ir), ut1 = __fmul_rn(U[2], ir), ut2 = __fmul_rn(U[3], ir);
#else
  const float un = U[1] * ir, ut1 = U[2] * ir, ut2 = U[3] * ir;
#endif
  const float ke = (0.5f * rho) * (un * un + (ut1 * ut1 + ut2 * ut2));
  const float eint = U[4] - ke;
  return (eint > float(kDualEta2) * U[4]) ? eint : U[5];
}

// Monotonised centred slope, zero at a local extremum.
template <typename T>
CELLO_HD T limited_slope(T am, T a0, T ap) {
  T dl = a0 - am;
  T dr = ap - a0;
  T da = T(0.5) * (ap - am);
  T m = vmin(vabs(da), vmin(T(2) * vabs(dl), T(2) * vabs(dr)));
  return (dl * dr > T(0)) ? vcopysign(m, da) : T(0);
}

// Interface value between cells j and j+1 in limited form.
template <typename T>
CELLO_HD T interface_value(T a0, T a1, T dm0, T dm1) {
  return T(0.5) * (a0 + a1) - (dm1 - dm0) * T(1.0 / 6.0);
}

// Shock detector of the flattening coefficient.
template <typename T>
CELLO_HD T flatten_tilde(T pm2, T pm1, T pp1, T pp2, T um1, T up1) {
  T dp1 = pp1 - pm1;
  T dp2 = pp2 - pm2;
  bool shock = (vabs(dp1) > T(kEpsShock) * vmin(pp1, pm1)) && (um1 - up1 > T(0)) && (dp2 != T(0));
  T ratio = vdiv(dp1, (dp2 != T(0)) ? dp2 : T(1));
  T ft = vmax(vmin(T(kOmega2) * (ratio - T(kOmega1)), T(1)), T(0));
  return shock ? ft : T(0);
}

// Contact-steepening weight of a cell (Colella & Woodward 1984, Sec. 1 on a
// uniform grid, with the gas-dynamics condition of their Sec. 3): from the
// densities of cells j-2 .. j+2 and the pressures of cells j-1, j+1, with
// second differences D, eta~ = -(D_{j+1} - D_{j-1}) / (6 (rho_{j+1} -
// rho_{j-1})), zero where the D have one sign, where the density jump is
// below 1 % or where the relative pressure jump exceeds gamma K0 times the
// relative density jump; eta = clamp(20 (eta~ - 0.05), 0, 1).
constexpr double kEpsSteep = 0.01;
constexpr double kEta1 = 20.0, kEta2 = 0.05;
constexpr double kK0Steep = 0.1;

template <typename T>
CELLO_HD T steepening_eta(T rm2, T rm1, T r0, T rp1, T rp2, T pm1, T pp1, T gamma) {
  const T Dm = (r0 - T(2) * rm1) + rm2;
  const T Dp = (rp2 - T(2) * rp1) + r0;
  const T drho = rp1 - rm1;
  const bool off = (Dp * Dm > T(0)) || (vabs(drho) - T(kEpsSteep) * vmin(vabs(rp1), vabs(rm1)) < T(0)) ||
                   (vdiv((gamma * T(kK0Steep)) * vabs(drho), vmin(rp1, rm1)) < vdiv(vabs(pp1 - pm1), vmin(pp1, pm1)));
  const T eta_t = off ? T(0) : vdiv(-(Dp - Dm), T(6) * drho);
  return vmax(vmin(T(kEta1) * (eta_t - T(kEta2)), T(1)), T(0));
}

// Flatten towards the cell value, then apply the monotonicity constraints.
template <typename T>
CELLO_HD void flatten_monotone(T a, T f, T& aL, T& aR) {
  T l = f * a + (T(1) - f) * aL;
  T r = f * a + (T(1) - f) * aR;
  bool ext = (r - a) * (a - l) <= T(0);
  T da = r - l;
  T dm = a - T(0.5) * (l + r);
  T t1 = da * dm;
  T t2 = (da * da) * T(1.0 / 6.0);
  aL = ext ? a : ((t1 > t2) ? T(3) * a - T(2) * r : l);
  aR = ext ? a : ((-t2 > t1) ? T(3) * a - T(2) * l : r);
}

template <typename T>
CELLO_HD T avg_right(T aL, T aR, T a6, T s) {
  T da = aR - aL;
  return aR - (T(0.5) * s) * (da - (T(1) - T(2.0 / 3.0) * s) * a6);
}

template <typename T>
CELLO_HD T avg_left(T aL, T aR, T a6, T s) {
  T da = aR - aL;
  return aL + (T(0.5) * s) * (da + (T(1) - T(2.0 / 3.0) * s) * a6);
}

// Characteristic tracing of one cell to its two edges at the half step.
// W = cell-centre primitives, aL/aR = monotone edge values; outputs the state
// at the left edge (Wm, right state of interface j-1/2) and at the right edge
// (Wp, left state of interface j+1/2).  NQ = 6: the specific internal energy
// of the dual-energy formalism rides the entropy wave like the transverse
// velocities.
template <typename T, int NQ = 5>
CELLO_HD void trace(const T W[NQ], const T aL[NQ], const T aR[NQ], T dtdx,
                                      const Gas<T>& gs, T Wm[NQ], T Wp[NQ]) {
  const T rho = W[0], un = W[1], p = W[4];
  const T csq = vdiv(gs.gamma * p, rho);
  const T c = vsqrt(csq);
  T a6[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) a6[q] = T(6) * (W[q] - T(0.5) * (aL[q] + aR[q]));
  const T lm = un - c, l0 = un, lp = un + c;
  const T half_rho_c = vdiv(T(0.5) * rho, c);
  const T half_inv_csq = vdiv(T(0.5), csq);
  const T c_rho = vdiv(c, rho);

  {  // right edge: waves moving right
    const T sp = lp * dtdx, s0 = l0 * dtdx, sm = lm * dtdx;
    T ref[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) ref[q] = (lp > T(0)) ? avg_right(aL[q], aR[q], a6[q], sp) : aR[q];
    T bm = T(0), b0 = T(0);
    if (lm > T(0))
      bm = (ref[4] - avg_right(aL[4], aR[4], a6[4], sm)) * half_inv_csq -
           (ref[1] - avg_right(aL[1], aR[1], a6[1], sm)) * half_rho_c;
    if (l0 > T(0))
      b0 = (ref[0] - avg_right(aL[0], aR[0], a6[0], s0)) - vdiv(ref[4] - avg_right(aL[4], aR[4], a6[4], s0), csq);
    Wp[0] = vmax(ref[0] - (b0 + bm), T(kRhoFloor));
    Wp[1] = ref[1] + c_rho * bm;
    Wp[4] = vmax(ref[4] - csq * bm, T(kPFloor));
    Wp[2] = (l0 > T(0)) ? avg_right(aL[2], aR[2], a6[2], s0) : ref[2];
    Wp[3] = (l0 > T(0)) ? avg_right(aL[3], aR[3], a6[3], s0) : ref[3];
#pragma unroll
    for (int q = 5; q < NQ; ++q) Wp[q] = (l0 > T(0)) ? avg_right(aL[q], aR[q], a6[q], s0) : ref[q];
  }
  {  // left edge: waves moving left
    const T tm = -lm * dtdx, t0 = -l0 * dtdx, tp = -lp * dtdx;
    T ref[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) ref[q] = (lm < T(0)) ? avg_left(aL[q], aR[q], a6[q], tm) : aL[q];
    T bp = T(0), b0 = T(0);
    if (lp < T(0))
      bp = (ref[4] - avg_left(aL[4], aR[4], a6[4], tp)) * half_inv_csq +
           (ref[1] - avg_left(aL[1], aR[1], a6[1], tp)) * half_rho_c;
    if (l0 < T(0))
      b0 = (ref[0] - avg_left(aL[0], aR[0], a6[0], t0)) - vdiv(ref[4] - avg_left(aL[4], aR[4], a6[4], t0), csq);
    Wm[0] = vmax(ref[0] - (b0 + bp), T(kRhoFloor));
    Wm[1] = ref[1] - c_rho * bp;
    Wm[4] = vmax(ref[4] - csq * bp, T(kPFloor));
    Wm[2] = (l0 < T(0)) ? avg_left(aL[2], aR[2], a6[2], t0) : ref[2];
    Wm[3] = (l0 < T(0)) ? avg_left(aL[3], aR[3], a6[3], t0) : ref[3];
#pragma unroll
    for (int q = 5; q < NQ; ++q) Wm[q] = (l0 < T(0)) ? avg_left(aL[q], aR[q], a6[q], t0) : ref[q];
  }
}

// Two-shock approximate Riemann solver (Colella & Woodward 1984): fixed
// Newton steps on p* along shock curves on both sides (a lane whose p* stops
// changing leaves the loop early, which gives bit-identical results), u* the Z-weighted
// mean, sampled at x/t = 0 (u* >= 0 takes the left side), linear in a
// rarefaction fan between head and tail.  Fluxes (rho, m_n, m_t1, m_t2, E);
// NQ = 6 adds the flux of rho e (mass flux times the e of the sampled side)
// and uf, the normal velocity of the sampled state.
template <typename T, int NQ = 5>
CELLO_HD void riemann_flux(const T L[NQ], const T R[NQ], const Gas<T>& gs, T F[NQ], T* uf = nullptr) {
  const T rL = L[0], uL = L[1], pL = L[4];
  const T rR = R[0], uR = R[1], pR = R[4];
  const T CL = vsqrt((gs.gamma * pL) * rL);
  const T CR = vsqrt((gs.gamma * pR) * rR);
  T ps = ((CR * pL + CL * pR) + (CL * CR) * (uL - uR)) / (CL + CR);
  ps = vmax(ps, T(kPFloor));
  T WLs, WRs, uLs, uRs, ZL, ZR;
#pragma unroll 1
  for (int it = 0; it <= kRiemannIters; ++it) {
    WLs = CL * vsqrt(T(1) + gs.g1 * (ps / pL - T(1)));
    WRs = CR * vsqrt(T(1) + gs.g1 * (ps / pR - T(1)));
    uLs = uL - (ps - pL) / WLs;
    uRs = uR + (ps - pR) / WRs;
    ZL = ((T(2) * WLs) * WLs) * WLs / (WLs * WLs + CL * CL);
    ZR = ((T(2) * WRs) * WRs) * WRs / (WRs * WRs + CR * CR);
    if (it == kRiemannIters) break;
    const T pn = vmax(ps - ((ZL * ZR) * (uRs - uLs)) / (ZL + ZR), T(kPFloor));
    if (pn == ps) break;   // fixed point: every remaining step would repeat this one exactly
    ps = pn;
  }
  const T us = (ZL * uLs + ZR * uRs) / (ZL + ZR);

  const bool left = us >= T(0);
  const T rs = left ? rL : rR;
  const T u_s = left ? uL : uR;
  const T p_s = left ? pL : pR;
  const T W_s = left ? WLs : WRs;
  const T t1 = left ? L[2] : R[2];
  const T t2 = left ? L[3] : R[3];
  const T v_s = left ? -uL : uR;
  const T v_star = left ? -us : us;
  const T tau = T(1) / rs - (ps - p_s) / (W_s * W_s);
  T rstar = (tau > T(0)) ? T(1) / tau : T(kRhoFloor);
  rstar = vmax(rstar, T(kRhoFloor));
  const T c_s = vsqrt((gs.gamma * p_s) / rs);
  const T c_star = vsqrt((gs.gamma * ps) / rstar);
  const bool shock = ps > p_s;
  const T head = shock ? v_s + W_s / rs : v_s + c_s;
  const T tail = shock ? head : v_star + c_star;
  const bool orig = head <= T(0);
  const bool star = !orig && (tail > T(0));
  T r, u, p;
  if (orig) {
    r = rs; u = u_s; p = p_s;
  } else if (star) {
    r = rstar; u = us; p = ps;
  } else {
    const T w = head / (head - tail);
    r = rs + w * (rstar - rs);
    u = u_s + w * (us - u_s);
    p = p_s + w * (ps - p_s);
  }
  const T f0 = r * u;
  F[0] = f0;
  F[1] = f0 * u + p;
  F[2] = f0 * t1;
  F[3] = f0 * t2;
  const T E = p * gs.inv_gm1 + (T(0.5) * r) * (u * u + (t1 * t1 + t2 * t2));
  F[4] = u * (E + p);
  if constexpr (NQ > 5) {
    F[5] = f0 * (left ? L[5] : R[5]);
    *uf = u;
  }
}

// HLLC flux (Toro, Spruce & Speares 1994; Toro, Riemann Solvers and
// Numerical Methods, Sec. 10.4): Davis wave-speed bounds, contact speed S*,
// and the flux of the fan region at x/t = 0 (F_L if S_L >= 0, F*_L if
// S* >= 0, F*_R if S_R > 0, else F_R) with F*_K = F_K + S_K (U*_K - U_K),
// U*_K = m_K / (S_K - S*) (1, S*, v_K, w_K, E_K / rho_K + (S* - u_K)(S* +
// p_K / m_K)), m_K = rho_K (S_K - u_K).  Only the side that is sampled is
// evaluated past the wave speeds; each quantity is the same expression in
// the same order as a full evaluation of both sides.  NQ = 6: rho e is
// passive like the transverse momenta (flux rho u e, star value m_K / (S_K
// - S*) e_K), and uf is the normal velocity of the sampled region's state
// (u_K outside the fan, S* inside).
template <typename T, int NQ = 5>
CELLO_HD void hllc_flux(const T L[NQ], const T R[NQ], const Gas<T>& gs, T F[NQ], T* uf = nullptr) {
  const T rL = L[0], uL = L[1], pL = L[4];
  const T rR = R[0], uR = R[1], pR = R[4];
  const T cL = vsqrt(vdiv(gs.gamma * pL, rL));
  const T cR = vsqrt(vdiv(gs.gamma * pR, rR));
  const T SL = vmin(uL - cL, uR - cR);
  const T SR = vmax(uL + cL, uR + cR);
  const T mL = rL * (SL - uL);
  const T mR = rR * (SR - uR);
  const T Ss = vdiv((pR - pL) + (mL * uL - mR * uR), mL - mR);
  const bool left = (SL >= T(0)) || (Ss >= T(0));
  const T r = left ? rL : rR, u = left ? uL : uR, v = left ? L[2] : R[2], w = left ? L[3] : R[3];
  const T p = left ? pL : pR, S = left ? SL : SR, m = left ? mL : mR;
  const T E = p * gs.inv_gm1 + (T(0.5) * r) * (u * u + (v * v + w * w));
  const T f0 = r * u;
  F[0] = f0;
  F[1] = f0 * u + p;
  F[2] = f0 * v;
  F[3] = f0 * w;
  F[4] = u * (E + p);
  const bool outer = left ? (SL >= T(0)) : !(SR > T(0));
  T e = T(0);
  if constexpr (NQ > 5) {
    e = left ? L[5] : R[5];
    F[5] = f0 * e;
    *uf = outer ? u : Ss;
  }
  if (!outer) {
    const T fac = vdiv(m, S - Ss);
    const T Us[5] = {fac, fac * Ss, fac * v, fac * w, fac * (vdiv(E, r) + (Ss - u) * (Ss + vdiv(p, m)))};
    const T Uc[5] = {r, r * u, r * v, r * w, E};
#pragma unroll
    for (int k = 0; k < 5; ++k) F[k] = F[k] + S * (Us[k] - Uc[k]);
    if constexpr (NQ > 5) F[5] = F[5] + S * (fac * e - r * e);
  }
}

template <typename T>
CELLO_HD void riemann_flux_bulk(const T L[5], const T R[5], const Gas<T>& gs, T F[5]) {
  riemann_flux(L, R, gs, F);
}

// Six-component (dual-energy) form with the interface velocity.
template <typename T>
CELLO_HD void riemann_flux_bulk6(const T L[6], const T R[6], const Gas<T>& gs, T F[6], T* uf) {
  riemann_flux<T, 6>(L, R, gs, F, uf);
}

}  // namespace cello
