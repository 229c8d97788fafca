// Hand-written reverse mode of the per-interface PPM flux (the adjoint of
// the hydro Method of Sec. II.C with dt held fixed).  Each *_bwd function
// recomputes what it needs of its forward counterpart in ppm.cuh and
// accumulates the adjoints of its inputs (+=).  At a kink (min, max, a
// branch) the derivative of the branch the forward pass took is used.
#pragma once

#include "ppm.cuh"

namespace cello {

template <typename T>
CELLO_HD void to_primitive_bwd(const T U[5], const Gas<T>& gs, const T Wb[5], T Ub[5]) {
  const T rho = vmax(U[0], T(kRhoFloor));
  const T un = U[1] / rho, ut1 = U[2] / rho, ut2 = U[3] / rho;
  const T s = un * un + (ut1 * ut1 + ut2 * ut2);
  const T h = T(0.5) * rho;
  const T praw = gs.gm1 * (U[4] - h * s);
  const T prawb = (praw > T(kPFloor)) ? Wb[4] : T(0);
  Ub[4] += gs.gm1 * prawb;
  const T keb = -gs.gm1 * prawb;
  T rhob = Wb[0] + T(0.5) * (keb * s);
  const T sb = keb * h;
  const T unb = Wb[1] + T(2) * un * sb;
  const T t1b = Wb[2] + T(2) * ut1 * sb;
  const T t2b = Wb[3] + T(2) * ut2 * sb;
  Ub[1] += unb / rho;
  Ub[2] += t1b / rho;
  Ub[3] += t2b / rho;
  rhob -= (unb * un + t1b * ut1 + t2b * ut2) / rho;
  if (U[0] > T(kRhoFloor)) Ub[0] += rhob;
}

template <typename T>
CELLO_HD void limited_slope_bwd(T am, T a0, T ap, T ob, T& amb, T& a0b, T& apb) {
  const T dl = a0 - am, dr = ap - a0, da = T(0.5) * (ap - am);
  if (!(dl * dr > T(0))) return;
  const T mb = (da < T(0)) ? -ob : ob;
  const T adl = T(2) * vabs(dl), adr = T(2) * vabs(dr);
  const T inner = vmin(adl, adr);
  if (vabs(da) < inner) {
    const T dab = (da < T(0)) ? -mb : mb;
    apb += T(0.5) * dab;
    amb -= T(0.5) * dab;
  } else if (adl < adr) {
    const T dlb = T(2) * ((dl < T(0)) ? -mb : mb);
    a0b += dlb;
    amb -= dlb;
  } else {
    const T drb = T(2) * ((dr < T(0)) ? -mb : mb);
    apb += drb;
    a0b -= drb;
  }
}

template <typename T>
CELLO_HD void interface_value_bwd(T ob, T& a0b, T& a1b, T& dm0b, T& dm1b) {
  a0b += T(0.5) * ob;
  a1b += T(0.5) * ob;
  dm1b -= ob * T(1.0 / 6.0);
  dm0b += ob * T(1.0 / 6.0);
}

template <typename T>
CELLO_HD void flatten_tilde_bwd(T pm2, T pm1, T pp1, T pp2, T um1, T up1, T ob, T& pm2b, T& pm1b, T& pp1b,
                                T& pp2b) {
  const T dp1 = pp1 - pm1, dp2 = pp2 - pm2;
  const bool shock = (vabs(dp1) > T(kEpsShock) * vmin(pp1, pm1)) && (um1 - up1 > T(0)) && (dp2 != T(0));
  if (!shock) return;
  const T ratio = dp1 / dp2;
  const T x = T(kOmega2) * (ratio - T(kOmega1));
  if (!(x < T(1)) || !(x > T(0))) return;
  const T rb = T(kOmega2) * ob;
  const T dp1b = rb / dp2, dp2b = -(rb * ratio) / dp2;
  pp1b += dp1b;
  pm1b -= dp1b;
  pp2b += dp2b;
  pm2b -= dp2b;
}

template <typename T>
CELLO_HD void flatten_monotone_bwd(T a, T f, T aL, T aR, T oLb, T oRb, T& ab, T& fb, T& aLb, T& aRb) {
  const T l = f * a + (T(1) - f) * aL;
  const T r = f * a + (T(1) - f) * aR;
  const bool ext = (r - a) * (a - l) <= T(0);
  T lb = T(0), rb = T(0);
  if (ext) {
    ab += oLb + oRb;
  } else {
    const T da = r - l, dm = a - T(0.5) * (l + r);
    const T t1 = da * dm, t2 = (da * da) * T(1.0 / 6.0);
    if (t1 > t2) {
      ab += T(3) * oLb;
      rb -= T(2) * oLb;
    } else {
      lb += oLb;
    }
    if (-t2 > t1) {
      ab += T(3) * oRb;
      lb -= T(2) * oRb;
    } else {
      rb += oRb;
    }
  }
  fb += lb * (a - aL) + rb * (a - aR);
  ab += (lb + rb) * f;
  aLb += lb * (T(1) - f);
  aRb += rb * (T(1) - f);
}

template <typename T>
CELLO_HD void avg_right_bwd(T aL, T aR, T a6, T s, T ob, T& aLb, T& aRb, T& a6b, T& sb) {
  const T h = T(0.5) * s, g = T(1) - T(2.0 / 3.0) * s;
  const T inner = (aR - aL) - g * a6;
  aRb += ob * (T(1) - h);
  aLb += ob * h;
  a6b += ob * (h * g);
  sb -= ob * (T(0.5) * inner + h * (T(2.0 / 3.0) * a6));
}

template <typename T>
CELLO_HD void avg_left_bwd(T aL, T aR, T a6, T s, T ob, T& aLb, T& aRb, T& a6b, T& sb) {
  const T h = T(0.5) * s, g = T(1) - T(2.0 / 3.0) * s;
  const T inner = (aR - aL) + g * a6;
  aLb += ob * (T(1) - h);
  aRb += ob * h;
  a6b += ob * (h * g);
  sb += ob * (T(0.5) * inner - h * (T(2.0 / 3.0) * a6));
}

// Reverse of trace(): adjoints of the two edge states -> adjoints of the
// cell-centre primitives and of the monotone edge values.
template <typename T>
CELLO_HD void trace_bwd(const T W[5], const T aL[5], const T aR[5], T dtdx, const Gas<T>& gs, const T Wmb[5],
                        const T Wpb[5], T Wb[5], T aLb[5], T aRb[5]) {
  const T rho = W[0], un = W[1], p = W[4];
  const T csq = (gs.gamma * p) / rho;
  const T c = vsqrt(csq);
  T a6[5], a6b[5];
  for (int q = 0; q < 5; ++q) {
    a6[q] = T(6) * (W[q] - T(0.5) * (aL[q] + aR[q]));
    a6b[q] = T(0);
  }
  const T lm = un - c, l0 = un, lp = un + c;
  const T hrc = (T(0.5) * rho) / c;
  const T hic = T(0.5) / csq;
  const T cr = c / rho;
  T lmb = 0, l0b = 0, lpb = 0, csqb = 0, cb = 0, rhob = 0, hrcb = 0, hicb = 0, crb = 0;

  {  // right edge
    const T sp = lp * dtdx, s0 = l0 * dtdx, sm = lm * dtdx;
    T ref[5], refb[5];
    for (int q = 0; q < 5; ++q) {
      ref[q] = (lp > T(0)) ? avg_right(aL[q], aR[q], a6[q], sp) : aR[q];
      refb[q] = T(0);
    }
    T bm = T(0), b0 = T(0), B1 = T(0), B4 = T(0), A0 = T(0), A4 = T(0);
    if (lm > T(0)) {
      B4 = avg_right(aL[4], aR[4], a6[4], sm);
      B1 = avg_right(aL[1], aR[1], a6[1], sm);
      bm = (ref[4] - B4) * hic - (ref[1] - B1) * hrc;
    }
    if (l0 > T(0)) {
      A0 = avg_right(aL[0], aR[0], a6[0], s0);
      A4 = avg_right(aL[4], aR[4], a6[4], s0);
      b0 = (ref[0] - A0) - (ref[4] - A4) / csq;
    }
    T bmb = 0, b0b = 0, spb = 0, s0b = 0, smb = 0;
    // transverse components
    for (int q = 2; q < 4; ++q) {
      if (l0 > T(0)) avg_right_bwd(aL[q], aR[q], a6[q], s0, Wpb[q], aLb[q], aRb[q], a6b[q], s0b);
      else refb[q] += Wpb[q];
    }
    {  // Wp[4] = max(ref4 - csq*bm, floor)
      const T x4 = ref[4] - csq * bm;
      if (x4 > T(kPFloor)) {
        refb[4] += Wpb[4];
        csqb -= Wpb[4] * bm;
        bmb -= Wpb[4] * csq;
      }
    }
    refb[1] += Wpb[1];  // Wp[1] = ref1 + cr*bm
    crb += Wpb[1] * bm;
    bmb += Wpb[1] * cr;
    {  // Wp[0] = max(ref0 - (b0 + bm), floor)
      const T x0 = ref[0] - (b0 + bm);
      if (x0 > T(kRhoFloor)) {
        refb[0] += Wpb[0];
        b0b -= Wpb[0];
        bmb -= Wpb[0];
      }
    }
    if (l0 > T(0)) {
      refb[0] += b0b;
      const T A0b = -b0b;
      const T D4 = ref[4] - A4;
      const T D4b = -b0b / csq;
      csqb += b0b * D4 / (csq * csq);
      refb[4] += D4b;
      const T A4b = -D4b;
      avg_right_bwd(aL[0], aR[0], a6[0], s0, A0b, aLb[0], aRb[0], a6b[0], s0b);
      avg_right_bwd(aL[4], aR[4], a6[4], s0, A4b, aLb[4], aRb[4], a6b[4], s0b);
    }
    if (lm > T(0)) {
      refb[4] += bmb * hic;
      hicb += bmb * (ref[4] - B4);
      refb[1] -= bmb * hrc;
      hrcb -= bmb * (ref[1] - B1);
      avg_right_bwd(aL[4], aR[4], a6[4], sm, -bmb * hic, aLb[4], aRb[4], a6b[4], smb);
      avg_right_bwd(aL[1], aR[1], a6[1], sm, bmb * hrc, aLb[1], aRb[1], a6b[1], smb);
    }
    for (int q = 0; q < 5; ++q) {
      if (lp > T(0)) avg_right_bwd(aL[q], aR[q], a6[q], sp, refb[q], aLb[q], aRb[q], a6b[q], spb);
      else aRb[q] += refb[q];
    }
    lpb += spb * dtdx;
    l0b += s0b * dtdx;
    lmb += smb * dtdx;
  }
  {  // left edge
    const T tm = -lm * dtdx, t0 = -l0 * dtdx, tp = -lp * dtdx;
    T ref[5], refb[5];
    for (int q = 0; q < 5; ++q) {
      ref[q] = (lm < T(0)) ? avg_left(aL[q], aR[q], a6[q], tm) : aL[q];
      refb[q] = T(0);
    }
    T bp = T(0), b0 = T(0), B1 = T(0), B4 = T(0), A0 = T(0), A4 = T(0);
    if (lp < T(0)) {
      B4 = avg_left(aL[4], aR[4], a6[4], tp);
      B1 = avg_left(aL[1], aR[1], a6[1], tp);
      bp = (ref[4] - B4) * hic + (ref[1] - B1) * hrc;
    }
    if (l0 < T(0)) {
      A0 = avg_left(aL[0], aR[0], a6[0], t0);
      A4 = avg_left(aL[4], aR[4], a6[4], t0);
      b0 = (ref[0] - A0) - (ref[4] - A4) / csq;
    }
    T bpb = 0, b0b = 0, tpb = 0, t0b = 0, tmb = 0;
    for (int q = 2; q < 4; ++q) {
      if (l0 < T(0)) avg_left_bwd(aL[q], aR[q], a6[q], t0, Wmb[q], aLb[q], aRb[q], a6b[q], t0b);
      else refb[q] += Wmb[q];
    }
    {
      const T x4 = ref[4] - csq * bp;
      if (x4 > T(kPFloor)) {
        refb[4] += Wmb[4];
        csqb -= Wmb[4] * bp;
        bpb -= Wmb[4] * csq;
      }
    }
    refb[1] += Wmb[1];  // Wm[1] = ref1 - cr*bp
    crb -= Wmb[1] * bp;
    bpb -= Wmb[1] * cr;
    {
      const T x0 = ref[0] - (b0 + bp);
      if (x0 > T(kRhoFloor)) {
        refb[0] += Wmb[0];
        b0b -= Wmb[0];
        bpb -= Wmb[0];
      }
    }
    if (l0 < T(0)) {
      refb[0] += b0b;
      const T A0b = -b0b;
      const T D4 = ref[4] - A4;
      const T D4b = -b0b / csq;
      csqb += b0b * D4 / (csq * csq);
      refb[4] += D4b;
      const T A4b = -D4b;
      avg_left_bwd(aL[0], aR[0], a6[0], t0, A0b, aLb[0], aRb[0], a6b[0], t0b);
      avg_left_bwd(aL[4], aR[4], a6[4], t0, A4b, aLb[4], aRb[4], a6b[4], t0b);
    }
    if (lp < T(0)) {
      refb[4] += bpb * hic;
      hicb += bpb * (ref[4] - B4);
      refb[1] += bpb * hrc;
      hrcb += bpb * (ref[1] - B1);
      avg_left_bwd(aL[4], aR[4], a6[4], tp, -bpb * hic, aLb[4], aRb[4], a6b[4], tpb);
      avg_left_bwd(aL[1], aR[1], a6[1], tp, -bpb * hrc, aLb[1], aRb[1], a6b[1], tpb);
    }
    for (int q = 0; q < 5; ++q) {
      if (lm < T(0)) avg_left_bwd(aL[q], aR[q], a6[q], tm, refb[q], aLb[q], aRb[q], a6b[q], tmb);
      else aLb[q] += refb[q];
    }
    lmb -= tmb * dtdx;
    l0b -= t0b * dtdx;
    lpb -= tpb * dtdx;
  }
  // shared coefficients
  T unb = lmb + l0b + lpb;
  cb += lpb - lmb;
  rhob += T(0.5) * hrcb / c;
  cb -= hrcb * hrc / c;
  csqb -= hicb * hic / csq;
  cb += crb / rho;
  rhob -= crb * cr / rho;
  for (int q = 0; q < 5; ++q) {
    Wb[q] += T(6) * a6b[q];
    aLb[q] -= T(3) * a6b[q];
    aRb[q] -= T(3) * a6b[q];
  }
  csqb += cb / (T(2) * c);
  T pb = csqb * gs.gamma / rho;
  rhob -= csqb * csq / rho;
  Wb[0] += rhob;
  Wb[1] += unb;
  Wb[4] += pb;
}

// Shock-curve quantities of one side at pressure ps (as in riemann_flux).
template <typename T>
struct Curve {
  T x, W, us, Z;
};

template <typename T>
CELLO_HD Curve<T> curve(T ps, T pK, T CK, T uK, T sgn, const Gas<T>& gs) {
  Curve<T> c;
  c.x = T(1) + gs.g1 * (ps / pK - T(1));
  c.W = CK * vsqrt(c.x);
  c.us = (sgn < T(0)) ? uK - (ps - pK) / c.W : uK + (ps - pK) / c.W;
  c.Z = ((T(2) * c.W) * c.W) * c.W / (c.W * c.W + CK * CK);
  return c;
}

// Reverse of curve(): adjoints of (us, Z, W) -> (ps, pK, CK, uK).
template <typename T>
CELLO_HD void curve_bwd(T ps, T pK, T CK, T sgn, const Gas<T>& gs, const Curve<T>& c, T usb, T Zb, T Wb,
                        T& psb, T& pKb, T& CKb, T& uKb) {
  const T W = c.W;
  const T den = W * W + CK * CK;
  T Wbar = Wb + Zb * ((T(2) * W * W * W * W + T(6) * W * W * CK * CK) / (den * den));
  CKb += Zb * (-(T(4) * W * W * W * CK) / (den * den));
  uKb += usb;
  // us = uK -/+ (ps - pK)/W
  const T q = (ps - pK) / W;
  const T qb = (sgn < T(0)) ? -usb : usb;
  psb += qb / W;
  pKb -= qb / W;
  Wbar -= qb * q / W;
  // W = CK*sqrt(x), x = 1 + g1*(ps/pK - 1)
  const T sx = vsqrt(c.x);
  CKb += Wbar * sx;
  const T xb = Wbar * CK / (T(2) * sx);
  psb += xb * gs.g1 / pK;
  pKb -= xb * gs.g1 * ps / (pK * pK);
}

// Reverse of riemann_flux(): flux adjoints -> adjoints of the two states.
template <typename T>
CELLO_HD void riemann_flux_bwd(const T L[5], const T R[5], const Gas<T>& gs, const T Fb[5], T Lb[5], T Rb[5]) {
  const T rL = L[0], uL = L[1], pL = L[4];
  const T rR = R[0], uR = R[1], pR = R[4];
  const T CL = vsqrt((gs.gamma * pL) * rL);
  const T CR = vsqrt((gs.gamma * pR) * rR);
  T ps_hist[kRiemannIters + 1];
  bool floor_hit[kRiemannIters + 1];
  const T ps_raw0 = ((CR * pL + CL * pR) + (CL * CR) * (uL - uR)) / (CL + CR);
  T ps = vmax(ps_raw0, T(kPFloor));
  floor_hit[0] = !(ps_raw0 > T(kPFloor));
  ps_hist[0] = ps;
  for (int it = 0; it < kRiemannIters; ++it) {
    const Curve<T> cl = curve(ps, pL, CL, uL, T(-1), gs), cr = curve(ps, pR, CR, uR, T(1), gs);
    const T raw = ps - ((cl.Z * cr.Z) * (cr.us - cl.us)) / (cl.Z + cr.Z);
    ps = vmax(raw, T(kPFloor));
    floor_hit[it + 1] = !(raw > T(kPFloor));
    ps_hist[it + 1] = ps;
  }
  const Curve<T> cl = curve(ps, pL, CL, uL, T(-1), gs), cr = curve(ps, pR, CR, uR, T(1), gs);
  const T Dz = cl.Z + cr.Z;
  const T us = (cl.Z * cl.us + cr.Z * cr.us) / Dz;
  const bool left = us >= T(0);
  const T rs = left ? rL : rR, u_s = left ? uL : uR, p_s = left ? pL : pR, W_s = left ? cl.W : cr.W;
  const T t1 = left ? L[2] : R[2], t2 = left ? L[3] : R[3];
  const T v_s = left ? -uL : uR, v_star = left ? -us : us;
  const T tau = T(1) / rs - (ps - p_s) / (W_s * W_s);
  const T rstar_raw = (tau > T(0)) ? T(1) / tau : T(kRhoFloor);
  const T rstar = vmax(rstar_raw, T(kRhoFloor));
  const T c_s = vsqrt((gs.gamma * p_s) / rs);
  const T c_star = vsqrt((gs.gamma * ps) / rstar);
  const bool shock = ps > p_s;
  const T head = shock ? v_s + W_s / rs : v_s + c_s;
  const T tail = shock ? head : v_star + c_star;
  const bool orig = head <= T(0);
  const bool star = !orig && (tail > T(0));
  T r, u, p, w = T(0);
  if (orig) {
    r = rs; u = u_s; p = p_s;
  } else if (star) {
    r = rstar; u = us; p = ps;
  } else {
    w = head / (head - tail);
    r = rs + w * (rstar - rs);
    u = u_s + w * (us - u_s);
    p = p_s + w * (ps - p_s);
  }
  // flux
  const T f0 = r * u;
  const T E = p * gs.inv_gm1 + (T(0.5) * r) * (u * u + (t1 * t1 + t2 * t2));
  const T Eb = Fb[4] * u;
  const T f0b = Fb[0] + Fb[1] * u + Fb[2] * t1 + Fb[3] * t2;
  T ub = Fb[1] * f0 + Fb[4] * (E + p) + f0b * r + Eb * (T(0.5) * r) * (T(2) * u);
  T pb = Fb[1] + Fb[4] * u + Eb * gs.inv_gm1;
  T rb = f0b * u + Eb * (T(0.5) * (u * u + (t1 * t1 + t2 * t2)));
  const T t1b = Fb[2] * f0 + Eb * (T(0.5) * r) * (T(2) * t1);
  const T t2b = Fb[3] * f0 + Eb * (T(0.5) * r) * (T(2) * t2);
  // sampling
  T rsb = 0, u_sb = 0, p_sb = 0, W_sb = 0, rstarb = 0, usb = 0, psb = 0, v_sb = 0, v_starb = 0, c_sb = 0,
    c_starb = 0;
  if (orig) {
    rsb += rb; u_sb += ub; p_sb += pb;
  } else if (star) {
    rstarb += rb; usb += ub; psb += pb;
  } else {
    const T wb = rb * (rstar - rs) + ub * (us - u_s) + pb * (ps - p_s);
    rsb += rb * (T(1) - w); rstarb += rb * w;
    u_sb += ub * (T(1) - w); usb += ub * w;
    p_sb += pb * (T(1) - w); psb += pb * w;
    const T den = head - tail;
    const T headb = wb * (-tail) / (den * den);
    const T tailb = wb * head / (den * den);
    v_sb += headb; c_sb += headb;          // rarefaction: head = v_s + c_s
    v_starb += tailb; c_starb += tailb;    //              tail = v* + c*
  }
  {  // c_star = sqrt(gamma*ps/rstar)
    const T x = (gs.gamma * ps) / rstar;
    const T xb = c_starb / (T(2) * c_star);
    psb += xb * gs.gamma / rstar;
    rstarb -= xb * x / rstar;
  }
  {  // c_s = sqrt(gamma*p_s/rs)
    const T x = (gs.gamma * p_s) / rs;
    const T xb = c_sb / (T(2) * c_s);
    p_sb += xb * gs.gamma / rs;
    rsb -= xb * x / rs;
  }
  if (rstar_raw > T(kRhoFloor) && tau > T(0)) {  // rstar = 1/tau
    const T taub = -rstarb * rstar * rstar;
    rsb -= taub / (rs * rs);
    const T w2 = W_s * W_s;
    psb -= taub / w2;
    p_sb += taub / w2;
    W_sb += taub * T(2) * (ps - p_s) / (w2 * W_s);
  }
  T Lb_[5] = {0, 0, 0, 0, 0}, Rb_[5] = {0, 0, 0, 0, 0};
  if (left) {
    Lb_[0] += rsb; Lb_[1] += u_sb - v_sb; Lb_[4] += p_sb; Lb_[2] += t1b; Lb_[3] += t2b;
    usb -= v_starb;
  } else {
    Rb_[0] += rsb; Rb_[1] += u_sb + v_sb; Rb_[4] += p_sb; Rb_[2] += t1b; Rb_[3] += t2b;
    usb += v_starb;
  }
  // us = (ZL*usL + ZR*usR)/Dz
  T ZLb = usb * (cl.us - us) / Dz, ZRb = usb * (cr.us - us) / Dz;
  T usLb = usb * cl.Z / Dz, usRb = usb * cr.Z / Dz;
  T WLb = left ? W_sb : T(0), WRb = left ? T(0) : W_sb;
  T CLb = 0, CRb = 0;
  curve_bwd(ps, pL, CL, T(-1), gs, cl, usLb, ZLb, WLb, psb, Lb_[4], CLb, Lb_[1]);
  curve_bwd(ps, pR, CR, T(1), gs, cr, usRb, ZRb, WRb, psb, Rb_[4], CRb, Rb_[1]);
  // Newton iterations in reverse: ps_{k+1} = max(ps_k - q(ps_k), floor)
  for (int it = kRiemannIters - 1; it >= 0; --it) {
    if (floor_hit[it + 1]) {
      psb = T(0);
      continue;
    }
    const T pk = ps_hist[it];
    const Curve<T> a = curve(pk, pL, CL, uL, T(-1), gs), b = curve(pk, pR, CR, uR, T(1), gs);
    const T D = a.Z + b.Z, du = b.us - a.us;
    const T q = ((a.Z * b.Z) * du) / D;
    const T qb = -psb;   // psb of ps_k accumulates the direct term below
    const T aZb = qb * (b.Z * du - q) / D;
    const T bZb = qb * (a.Z * du - q) / D;
    const T dub = qb * (a.Z * b.Z) / D;
    T pkb = psb;
    curve_bwd(pk, pL, CL, T(-1), gs, a, -dub, aZb, T(0), pkb, Lb_[4], CLb, Lb_[1]);
    curve_bwd(pk, pR, CR, T(1), gs, b, dub, bZb, T(0), pkb, Rb_[4], CRb, Rb_[1]);
    psb = pkb;
  }
  if (!floor_hit[0]) {  // ps0 = ((CR pL + CL pR) + (CL CR)(uL - uR)) / (CL + CR)
    const T Dn = CL + CR;
    const T num = (CR * pL + CL * pR) + (CL * CR) * (uL - uR);
    const T nb = psb / Dn;
    const T Dnb = -psb * num / (Dn * Dn);
    Lb_[4] += nb * CR;
    Rb_[4] += nb * CL;
    CLb += nb * (pR + CR * (uL - uR)) + Dnb;
    CRb += nb * (pL + CL * (uL - uR)) + Dnb;
    Lb_[1] += nb * (CL * CR);
    Rb_[1] -= nb * (CL * CR);
  }
  // CK = sqrt(gamma*pK*rK)
  Lb_[4] += CLb * (gs.gamma * rL) / (T(2) * CL);
  Lb_[0] += CLb * (gs.gamma * pL) / (T(2) * CL);
  Rb_[4] += CRb * (gs.gamma * rR) / (T(2) * CR);
  Rb_[0] += CRb * (gs.gamma * pR) / (T(2) * CR);
  for (int q2 = 0; q2 < 5; ++q2) {
    Lb[q2] += Lb_[q2];
    Rb[q2] += Rb_[q2];
  }
}

// The flux at the interface between cells 3 and 4 of an 8-cell window of
// conserved states (sweep component order), and its vector-Jacobian
// product: Ub[c][k] += sum_q Fb[q] dF_q/dU[c][k].
template <typename T>
CELLO_HD void window_flux(const T U[8][5], T dtdx, const Gas<T>& gs, T F[5]) {
  T W[8][5];
  for (int c = 0; c < 8; ++c) to_primitive(U[c], gs, W[c]);
  T dm[8][5];
  for (int c = 1; c < 7; ++c)
    for (int q = 0; q < 5; ++q) dm[c][q] = limited_slope(W[c - 1][q], W[c][q], W[c + 1][q]);
  T ai[8][5];  // ai[c] = interface c|c+1, c = 2, 3, 4
  for (int c = 2; c < 5; ++c)
    for (int q = 0; q < 5; ++q) ai[c][q] = interface_value(W[c][q], W[c + 1][q], dm[c][q], dm[c + 1][q]);
  T ft[8];
  for (int c = 2; c < 6; ++c)
    ft[c] = flatten_tilde(W[c - 2][4], W[c - 1][4], W[c + 1][4], W[c + 2][4], W[c - 1][1], W[c + 1][1]);
  T edge[2][5];
  for (int side = 0; side < 2; ++side) {
    const int j = 3 + side;
    const T s = W[j + 1][4] - W[j - 1][4];
    const T f = (s > T(0)) ? vmax(ft[j], ft[j - 1]) : ((s < T(0)) ? vmax(ft[j], ft[j + 1]) : ft[j]);
    T aL[5], aR[5], Wm[5], Wp[5];
    for (int q = 0; q < 5; ++q) {
      aL[q] = ai[j - 1][q];
      aR[q] = ai[j][q];
      flatten_monotone(W[j][q], f, aL[q], aR[q]);
    }
    trace(W[j], aL, aR, dtdx, gs, Wm, Wp);
    for (int q = 0; q < 5; ++q) edge[side][q] = side == 0 ? Wp[q] : Wm[q];
  }
  riemann_flux(edge[0], edge[1], gs, F);
}

template <typename T>
CELLO_HD void window_flux_vjp(const T U[8][5], T dtdx, const Gas<T>& gs, const T Fb[5], T Ub[8][5]) {
  T W[8][5];
  for (int c = 0; c < 8; ++c) to_primitive(U[c], gs, W[c]);
  T dm[8][5];
  for (int c = 1; c < 7; ++c)
    for (int q = 0; q < 5; ++q) dm[c][q] = limited_slope(W[c - 1][q], W[c][q], W[c + 1][q]);
  T ai[8][5];
  for (int c = 2; c < 5; ++c)
    for (int q = 0; q < 5; ++q) ai[c][q] = interface_value(W[c][q], W[c + 1][q], dm[c][q], dm[c + 1][q]);
  T ft[8];
  for (int c = 2; c < 6; ++c)
    ft[c] = flatten_tilde(W[c - 2][4], W[c - 1][4], W[c + 1][4], W[c + 2][4], W[c - 1][1], W[c + 1][1]);
  T fval[2], aLm[2][5], aRm[2][5], edge[2][5];
  int fsel[2];  // -1: f = ft[j-1], 0: ft[j], +1: ft[j+1]
  for (int side = 0; side < 2; ++side) {
    const int j = 3 + side;
    const T s = W[j + 1][4] - W[j - 1][4];
    T f;
    if (s > T(0)) {
      f = vmax(ft[j], ft[j - 1]);
      fsel[side] = (ft[j] > ft[j - 1]) ? 0 : -1;
    } else if (s < T(0)) {
      f = vmax(ft[j], ft[j + 1]);
      fsel[side] = (ft[j] > ft[j + 1]) ? 0 : 1;
    } else {
      f = ft[j];
      fsel[side] = 0;
    }
    fval[side] = f;
    T Wm[5], Wp[5];
    for (int q = 0; q < 5; ++q) {
      aLm[side][q] = ai[j - 1][q];
      aRm[side][q] = ai[j][q];
      flatten_monotone(W[j][q], f, aLm[side][q], aRm[side][q]);
    }
    trace(W[j], aLm[side], aRm[side], dtdx, gs, Wm, Wp);
    for (int q = 0; q < 5; ++q) edge[side][q] = side == 0 ? Wp[q] : Wm[q];
  }
  // ---- reverse
  T eb[2][5] = {{0, 0, 0, 0, 0}, {0, 0, 0, 0, 0}};
  riemann_flux_bwd(edge[0], edge[1], gs, Fb, eb[0], eb[1]);
  T Wb[8][5], aib[8][5], dmb[8][5], ftb[8];
  for (int c = 0; c < 8; ++c) {
    ftb[c] = T(0);
    for (int q = 0; q < 5; ++q) Wb[c][q] = aib[c][q] = dmb[c][q] = T(0);
  }
  for (int side = 0; side < 2; ++side) {
    const int j = 3 + side;
    const T zero5[5] = {0, 0, 0, 0, 0};
    T aLb[5] = {0, 0, 0, 0, 0}, aRb[5] = {0, 0, 0, 0, 0};
    trace_bwd(W[j], aLm[side], aRm[side], dtdx, gs, side == 0 ? zero5 : eb[1], side == 0 ? eb[0] : zero5, Wb[j],
              aLb, aRb);
    T fb = T(0);
    for (int q = 0; q < 5; ++q)
      flatten_monotone_bwd(W[j][q], fval[side], ai[j - 1][q], ai[j][q], aLb[q], aRb[q], Wb[j][q], fb, aib[j - 1][q],
                           aib[j][q]);
    ftb[j + fsel[side]] += fb;
  }
  for (int c = 5; c >= 2; --c)
    flatten_tilde_bwd(W[c - 2][4], W[c - 1][4], W[c + 1][4], W[c + 2][4], W[c - 1][1], W[c + 1][1], ftb[c], Wb[c - 2][4],
                      Wb[c - 1][4], Wb[c + 1][4], Wb[c + 2][4]);
  for (int c = 4; c >= 2; --c)
    for (int q = 0; q < 5; ++q) interface_value_bwd(aib[c][q], Wb[c][q], Wb[c + 1][q], dmb[c][q], dmb[c + 1][q]);
  for (int c = 6; c >= 1; --c)
    for (int q = 0; q < 5; ++q) limited_slope_bwd(W[c - 1][q], W[c][q], W[c + 1][q], dmb[c][q], Wb[c - 1][q], Wb[c][q],
                                                  Wb[c + 1][q]);
  for (int c = 0; c < 8; ++c) to_primitive_bwd(U[c], gs, Wb[c], Ub[c]);
}

}  // namespace cello
