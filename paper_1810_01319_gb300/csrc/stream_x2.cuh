// Float32 arithmetic of the sweep in packed lane pairs.
//
// The FP32 pipe of sm_100-class GPUs executes two-lane add, multiply and
// fused multiply-add instructions (add / mul / fma / sub .rn.f32x2): one
// issue slot advances two values.  The sweep is bound by instruction issue,
// and most of its arithmetic applies one formula to every field of a cell
// (the limited slopes and interface values of Sec. II.C's PPM, flattening
// and the CW84 monotonicity constraints, the parabola averages of
// characteristic tracing, the conservative update).  Here a cell's fields
// are held in three groups that always pass through the same formulas:
//   A = (u_n, p)    B = (u_t1, u_t2)    C = rho, or (rho, e) with the
//                                         dual-energy formalism
// and each formula runs once per group; the two-shock Riemann solver
// evaluates its left and right shock curves as one pair.  Comparisons,
// minima, maxima and selects stay per lane (the FP32 pipe has no two-lane
// forms of them).
//
// Every float32 expression of the sweep is explicitly rounded: each add,
// multiply and fused multiply-add is written out (__fadd_rn, __fmaf_rn and
// their pair forms), none is left to the compiler's contraction.  A lane of
// a pair rounds exactly like the scalar operation, so the scalar group C of
// the five-field form and the pair (rho, e) of the six-field form give the
// same rho, and the streaming and shared-memory forms of the sweep, which
// both call these functions, compute the same bits.  The expressions follow
// the formulas of ppm.cuh term by term.
#pragma once

#include <type_traits>

#include "ppm.cuh"

namespace cello {
namespace px {

// ---- rounded operations on one value (float) or a lane pair (float2) ----
__device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

__device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub(float2 a, float2 b) {
  unsigned long long x, y, d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(y) : "f"(b.x), "f"(b.y));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(x), "l"(y));
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(d));
  return r;
}

template <class V> __device__ __forceinline__ V splat(float s);
template <> __device__ __forceinline__ float splat<float>(float s) { return s; }
template <> __device__ __forceinline__ float2 splat<float2>(float s) { return make_float2(s, s); }

// per-lane application of a scalar function
template <class Fn, class... A>
__device__ __forceinline__ float lanes(Fn f, float a, A... r) { return f(a, r...); }
template <class Fn, class... A>
__device__ __forceinline__ float2 lanes(Fn f, float2 a, A... r) { return make_float2(f(a.x, r.x...), f(a.y, r.y...)); }

__device__ __forceinline__ float lo(float a) { return a; }
__device__ __forceinline__ float lo(float2 a) { return a.x; }

// ---- a cell's fields in groups ----
template <int NQ>
struct Cell {
  using CT = typename std::conditional<NQ == 6, float2, float>::type;
  float2 a;   // (u_n, p), or the conserved / flux pair (m_n, E)
  float2 b;   // (u_t1, u_t2), or (m_t1, m_t2)
  CT c;       // rho (rho, e); or rho (rho, rho e)

  // field q of the sweep-local order (rho, n, t1, t2, E or p, rho e or e)
  __device__ __forceinline__ float get(int q) const {
    if (q == 0) return lo(c);
    if (q == 1) return a.x;
    if (q == 2) return b.x;
    if (q == 3) return b.y;
    if (q == 4) return a.y;
    if constexpr (NQ == 6) return c.y;
    return 0.0f;
  }
  __device__ __forceinline__ void set(int q, float v) {
    if (q == 0) {
      if constexpr (NQ == 6) c.x = v; else c = v;
    } else if (q == 1) a.x = v;
    else if (q == 2) b.x = v;
    else if (q == 3) b.y = v;
    else if (q == 4) a.y = v;
    else if constexpr (NQ == 6) c.y = v;
  }
};

template <int NQ, class Fn>
__device__ __forceinline__ Cell<NQ> each(Fn f, const Cell<NQ>& x) {
  Cell<NQ> r; r.a = f(x.a); r.b = f(x.b); r.c = f(x.c); return r;
}
template <int NQ, class Fn>
__device__ __forceinline__ Cell<NQ> each(Fn f, const Cell<NQ>& x, const Cell<NQ>& y) {
  Cell<NQ> r; r.a = f(x.a, y.a); r.b = f(x.b, y.b); r.c = f(x.c, y.c); return r;
}
template <int NQ, class Fn>
__device__ __forceinline__ Cell<NQ> each(Fn f, const Cell<NQ>& x, const Cell<NQ>& y, const Cell<NQ>& z) {
  Cell<NQ> r; r.a = f(x.a, y.a, z.a); r.b = f(x.b, y.b, z.b); r.c = f(x.c, y.c, z.c); return r;
}
template <int NQ, class Fn>
__device__ __forceinline__ Cell<NQ> each(Fn f, const Cell<NQ>& x, const Cell<NQ>& y, const Cell<NQ>& z,
                                         const Cell<NQ>& w) {
  Cell<NQ> r; r.a = f(x.a, y.a, z.a, w.a); r.b = f(x.b, y.b, z.b, w.b); r.c = f(x.c, y.c, z.c, w.c); return r;
}

// ---- per-field formulas (ppm.cuh), one group at a time ----

// Limited slope: dl = a0 - am, dr = ap - a0, da = (ap - am)/2; min(|da|,
// 2|dl|, 2|dr|) with the sign of da where dl dr > 0, else 0 (doubling is
// exact, so 2 min(|dl|, |dr|) equals min(2|dl|, 2|dr|)).
template <class V>
__device__ __forceinline__ V slope(V am, V a0, V ap) {
  const V dl = sub(a0, am), dr = sub(ap, a0);
  const V da = mul(splat<V>(0.5f), sub(ap, am));
  const V pr = mul(dl, dr);
  (void)pr;
  // with s = sign(da): s dl and s dr are both positive exactly where dl dr > 0
  const V sg = lanes([](float d) { return copysignf(1.0f, d); }, da);
  const V mn = mul(splat<V>(2.0f), lanes([](float x, float y) { return vmin(x, y); }, mul(sg, dl), mul(sg, dr)));
  return mul(sg, lanes([](float d, float m) { return vmax(vmin(fabsf(d), m), 0.0f); }, da, mn));
}

// Interface value (a0 + a1)/2 - (dm1 - dm0)/6.
template <class V>
__device__ __forceinline__ V interface_val(V a0, V a1, V dm0, V dm1) {
  return fma(sub(dm1, dm0), splat<V>(-1.0f / 6.0f), mul(splat<V>(0.5f), add(a0, a1)));
}

// Flattening towards the cell value (weights f, 1 - f) and the CW84
// monotonicity constraints.
template <class V>
__device__ __forceinline__ void flatten_mono(V a, V f, V omf, V& aL, V& aR) {
  const V fa = mul(f, a);
  const V l = fma(omf, aL, fa);
  const V r = fma(omf, aR, fa);
  const V ex = mul(sub(r, a), sub(a, l));                  // <= 0: local extremum
  const V da = sub(r, l);
  const V dm = fma(splat<V>(-0.5f), add(l, r), a);         // a - (l + r)/2
  const V t1 = mul(da, dm);
  const V t2 = mul(mul(da, da), splat<V>(1.0f / 6.0f));
  const V a3 = mul(splat<V>(3.0f), a);
  const V cl = fma(splat<V>(-2.0f), r, a3);                // 3a - 2r
  const V cr = fma(splat<V>(-2.0f), l, a3);                // 3a - 2l
  aL = lanes([](float e, float av, float u1, float u2, float c, float lv) {
               return (e <= 0.0f) ? av : ((u1 > u2) ? c : lv);
             },
             ex, a, t1, t2, cl, l);
  aR = lanes([](float e, float av, float u1, float u2, float c, float rv) {
               return (e <= 0.0f) ? av : ((-u2 > u1) ? c : rv);
             },
             ex, a, t1, t2, cr, r);
}

// Parabola average seen over a fraction s of the cell from its right edge,
// aR - (s/2)(da - (1 - 2s/3) a6), with nk = -(1 - 2s/3) and nh = -s/2 for
// the wave; from the left edge over a fraction t = -s, aL + (t/2)(da + (1 -
// 2t/3) a6) with kp = 1 + 2s/3 = 1 - 2t/3 and nh = t/2.
template <class V>
__device__ __forceinline__ V avg_r(V aR, V da, V a6, V nk, V nh) {
  return fma(nh, fma(nk, a6, da), aR);
}
template <class V>
__device__ __forceinline__ V avg_l(V aL, V da, V a6, V kp, V nh) {
  return fma(nh, fma(kp, a6, da), aL);
}

struct Wave {
  float2 nk, kp, nh;   // each the same value in both lanes
};

__device__ __forceinline__ Wave wave(float2 s) {
  Wave w;
  w.nk = fma(splat<float2>(2.0f / 3.0f), s, splat<float2>(-1.0f));
  w.kp = fma(splat<float2>(2.0f / 3.0f), s, splat<float2>(1.0f));
  w.nh = mul(splat<float2>(-0.5f), s);
  return w;
}

template <class V> __device__ __forceinline__ V pick(const float2& x);
template <> __device__ __forceinline__ float pick<float>(const float2& x) { return x.x; }
template <> __device__ __forceinline__ float2 pick<float2>(const float2& x) { return x; }

template <int NQ>
__device__ __forceinline__ Cell<NQ> avg_right(const Cell<NQ>& aR, const Cell<NQ>& da, const Cell<NQ>& a6,
                                              const Wave& w) {
  using CT = typename Cell<NQ>::CT;
  Cell<NQ> r;
  r.a = avg_r(aR.a, da.a, a6.a, w.nk, w.nh);
  r.b = avg_r(aR.b, da.b, a6.b, w.nk, w.nh);
  r.c = avg_r(aR.c, da.c, a6.c, pick<CT>(w.nk), pick<CT>(w.nh));
  return r;
}
template <int NQ>
__device__ __forceinline__ Cell<NQ> avg_left(const Cell<NQ>& aL, const Cell<NQ>& da, const Cell<NQ>& a6,
                                             const Wave& w) {
  using CT = typename Cell<NQ>::CT;
  Cell<NQ> r;
  r.a = avg_l(aL.a, da.a, a6.a, w.kp, w.nh);
  r.b = avg_l(aL.b, da.b, a6.b, w.kp, w.nh);
  r.c = avg_l(aL.c, da.c, a6.c, pick<CT>(w.kp), pick<CT>(w.nh));
  return r;
}

// Conserved -> primitive in groups (sweep-local conserved order in U).
template <int NQ>
__device__ __forceinline__ Cell<NQ> primitives(const float* U, const Gas<float>& gs) {
  Cell<NQ> W;
  const float rho = vmax(U[0], float(kRhoFloor));
  const float ir = __fdividef(1.0f, rho);
  const float un = mul(U[1], ir);
  W.b = mul(make_float2(U[2], U[3]), splat<float2>(ir));
  const float s = fma(un, un, fma(W.b.x, W.b.x, mul(W.b.y, W.b.y)));
  const float ke = mul(mul(0.5f, rho), s);
  float p;
  if constexpr (NQ == 6) {
    const float eint = sub(U[4], ke);
    const float src = (eint > mul(float(kDualEta1), U[4])) ? eint : U[5];
    p = vmax(mul(gs.gm1, src), float(kPFloor));
    W.c = make_float2(rho, mul(U[5], ir));
  } else {
    p = vmax(mul(gs.gm1, sub(U[4], ke)), float(kPFloor));
    W.c = rho;
  }
  W.a = make_float2(un, p);
  return W;
}

// Characteristic tracing of one cell (ppm.cuh: trace) in groups.
template <int NQ>
__device__ __forceinline__ void trace_cell(const Cell<NQ>& W, const Cell<NQ>& aL, const Cell<NQ>& aR, float2 dtdx2,
                                           const Gas<float>& gs, Cell<NQ>& Wm, Cell<NQ>& Wp) {
  const float rho = lo(W.c), un = W.a.x, p = W.a.y;
  const float csq = __fdividef(mul(gs.gamma, p), rho);
  const float c = sqrtf(csq);
  const Cell<NQ> a6 = each([](auto w, auto l, auto r) {
    using V = decltype(w);
    return mul(splat<V>(6.0f), fma(splat<V>(-0.5f), add(l, r), w));
  }, W, aL, aR);
  const Cell<NQ> da = each([](auto l, auto r) { return sub(r, l); }, aL, aR);
  const float lm = sub(un, c), l0 = un, lp = add(un, c);
  const float half_rho_c = __fdividef(mul(0.5f, rho), c);
  const float half_inv_csq = __fdividef(0.5f, csq);
  const float c_rho = __fdividef(c, rho);
  const float2 un2 = splat<float2>(un), c2 = splat<float2>(c);
  const Wave Wp_ = wave(mul(add(un2, c2), dtdx2));   // lambda+ = u + c
  const Wave W0_ = wave(mul(un2, dtdx2));             // lambda0 = u
  const Wave Wm_ = wave(mul(sub(un2, c2), dtdx2));   // lambda- = u - c

  {  // right edge: waves moving right
    const Cell<NQ> avp = avg_right(aR, da, a6, Wp_);
    const Cell<NQ> ref = (lp > 0.0f) ? avp : aR;
    float bm = 0.0f, b0 = 0.0f;
    if (lm > 0.0f) {
      const float2 d = sub(ref.a, avg_r(aR.a, da.a, a6.a, Wm_.nk, Wm_.nh));
      bm = fma(d.y, half_inv_csq, -mul(d.x, half_rho_c));
    }
    const Cell<NQ> av0 = avg_right(aR, da, a6, W0_);
    if (l0 > 0.0f) b0 = sub(sub(lo(ref.c), lo(av0.c)), __fdividef(sub(ref.a.y, av0.a.y), csq));
    Wp.a.x = fma(c_rho, bm, ref.a.x);
    Wp.a.y = vmax(fma(-csq, bm, ref.a.y), float(kPFloor));
    Wp.b = (l0 > 0.0f) ? av0.b : ref.b;
    if constexpr (NQ == 6) {
      Wp.c.x = vmax(sub(ref.c.x, add(b0, bm)), float(kRhoFloor));
      Wp.c.y = (l0 > 0.0f) ? av0.c.y : ref.c.y;
    } else {
      Wp.c = vmax(sub(ref.c, add(b0, bm)), float(kRhoFloor));
    }
  }
  {  // left edge: waves moving left
    const Cell<NQ> avm = avg_left(aL, da, a6, Wm_);
    const Cell<NQ> ref = (lm < 0.0f) ? avm : aL;
    float bp = 0.0f, b0 = 0.0f;
    if (lp < 0.0f) {
      const float2 d = sub(ref.a, avg_l(aL.a, da.a, a6.a, Wp_.kp, Wp_.nh));
      bp = fma(d.y, half_inv_csq, mul(d.x, half_rho_c));
    }
    const Cell<NQ> av0 = avg_left(aL, da, a6, W0_);
    if (l0 < 0.0f) b0 = sub(sub(lo(ref.c), lo(av0.c)), __fdividef(sub(ref.a.y, av0.a.y), csq));
    Wm.a.x = fma(-c_rho, bp, ref.a.x);
    Wm.a.y = vmax(fma(-csq, bp, ref.a.y), float(kPFloor));
    Wm.b = (l0 < 0.0f) ? av0.b : ref.b;
    if constexpr (NQ == 6) {
      Wm.c.x = vmax(sub(ref.c.x, add(b0, bp)), float(kRhoFloor));
      Wm.c.y = (l0 < 0.0f) ? av0.c.y : ref.c.y;
    } else {
      Wm.c = vmax(sub(ref.c, add(b0, bp)), float(kRhoFloor));
    }
  }
}

// Contact-steepening weight (ppm.cuh: steepening_eta), explicitly rounded.
__device__ __forceinline__ float steepening(float rm2, float rm1, float r0, float rp1, float rp2, float pm1,
                                            float pp1, float gamma) {
  const float Dm = add(sub(r0, mul(2.0f, rm1)), rm2);
  const float Dp = add(sub(rp2, mul(2.0f, rp1)), r0);
  const float drho = sub(rp1, rm1);
  const bool off = (mul(Dp, Dm) > 0.0f) ||
                   (sub(fabsf(drho), mul(float(kEpsSteep), vmin(fabsf(rp1), fabsf(rm1)))) < 0.0f) ||
                   (__fdividef(mul(mul(gamma, float(kK0Steep)), fabsf(drho)), vmin(rp1, rm1)) <
                    __fdividef(fabsf(sub(pp1, pm1)), vmin(pp1, pm1)));
  const float eta_t = off ? 0.0f : __fdividef(-sub(Dp, Dm), mul(6.0f, drho));
  return vmax(vmin(mul(float(kEta1), sub(eta_t, float(kEta2))), 1.0f), 0.0f);
}

// Synchronised rho e of an updated cell (ppm.cuh: dual_sync), explicitly
// rounded; the kinetic energy as in primitives().
__device__ __forceinline__ float dual_sync6(const float v[6]) {
  const float rho = vmax(v[0], float(kRhoFloor));
  const float ir = __fdividef(1.0f, rho);
  const float un = mul(v[1], ir);
  const float2 t = mul(make_float2(v[2], v[3]), splat<float2>(ir));
  const float ke = mul(mul(0.5f, rho), fma(un, un, fma(t.x, t.x, mul(t.y, t.y))));
  const float eint = sub(v[4], ke);
  return (eint > mul(float(kDualEta2), v[4])) ? eint : v[5];
}

// Flux of the state (r, u, t1, t2, p) sampled at an interface: (r u, r u^2
// + p, r u t1, r u t2, u (E + p)) in groups (a = (F_n, F_E), b = the
// transverse pair, c = F_rho).
template <int NQ>
__device__ __forceinline__ void sampled_flux(float r, float u, float p, float2 t, const Gas<float>& gs, Cell<NQ>& F,
                                             float& E) {
  const float f0 = mul(r, u);
  E = fma(p, gs.inv_gm1, mul(mul(0.5f, r), fma(u, u, fma(t.x, t.x, mul(t.y, t.y)))));
  F.a = make_float2(fma(f0, u, p), mul(u, add(E, p)));
  F.b = mul(splat<float2>(f0), t);
  if constexpr (NQ == 6) F.c.x = f0; else F.c = f0;
}

// Two-shock Riemann solver (ppm.cuh: riemann_flux, the same iteration and
// sampling), the left and right shock curves evaluated in one lane pair
// (L, R).  The shock-curve quantities are rewritten with shared
// reciprocals, algebraically identical to the literal formulas:
// x = 1 + g1 (p*/p - 1) = (g1/p) p* + (1 - g1), W = C sqrt(x),
// (p* - p)/W = (p* - p) rsqrt(x)/C, Z = 2W^3/(W^2 + C^2) = 2 W x/(x + 1),
// with C = sqrt(gamma p rho) = (gamma p rho) rsqrt(gamma p rho); the float64
// path keeps the literal formulas.
template <int NQ>
__device__ __forceinline__ void two_shock(const Cell<NQ>& Lc, const Cell<NQ>& Rc, const Gas<float>& gs, Cell<NQ>& F,
                                          float* uf) {
  const float rL = lo(Lc.c), uL = Lc.a.x, pL = Lc.a.y;
  const float rR = lo(Rc.c), uR = Rc.a.x, pR = Rc.a.y;
  const float2 r2 = make_float2(rL, rR), u2 = make_float2(uL, uR), p2 = make_float2(pL, pR);
  const float2 q = mul(mul(splat<float2>(gs.gamma), p2), r2);
  const float2 iC = make_float2(rsqrtf(q.x), rsqrtf(q.y));
  const float2 C = mul(q, iC);
  float ps = __fdividef(fma(mul(C.x, C.y), sub(uL, uR), fma(C.y, pL, mul(C.x, pR))), add(C.x, C.y));
  ps = vmax(ps, float(kPFloor));
  const float2 a = make_float2(__fdividef(gs.g1, pL), __fdividef(gs.g1, pR));
  const float2 b = splat<float2>(1.0f - gs.g1);
  const float2 niC = mul(iC, make_float2(-1.0f, 1.0f));   // (-1/C_L, 1/C_R)
  float2 W, us, Z;
#pragma unroll 1
  for (int it = 0; it <= kRiemannIters; ++it) {
    const float2 ps2 = splat<float2>(ps);
    const float2 x = fma(a, ps2, b);                        // 1 + g1 (p*/p - 1)
    const float2 rx = make_float2(rsqrtf(x.x), rsqrtf(x.y));
    W = mul(C, mul(x, rx));                                 // C sqrt(x)
    us = fma(sub(ps2, p2), mul(niC, rx), u2);               // u_L - (p* - p_L)/W_L, u_R + (p* - p_R)/W_R
    const float2 num = mul(mul(splat<float2>(2.0f), W), x);
    const float2 den = add(x, splat<float2>(1.0f));
    Z = make_float2(__fdividef(num.x, den.x), __fdividef(num.y, den.y));
    if (it == kRiemannIters) break;
    const float pn =
        vmax(sub(ps, __fdividef(mul(mul(Z.x, Z.y), sub(us.y, us.x)), add(Z.x, Z.y))), float(kPFloor));
    if (pn == ps) break;   // fixed point (see riemann_flux)
    ps = pn;
  }
  const float ust = __fdividef(fma(Z.x, us.x, mul(Z.y, us.y)), add(Z.x, Z.y));
  const bool left = ust >= 0.0f;
  const float rs = left ? rL : rR;
  const float u_s = left ? uL : uR;
  const float p_s = left ? pL : pR;
  const float W_s = left ? W.x : W.y;
  const float2 t = left ? Lc.b : Rc.b;
  const float v_s = left ? -uL : uR;
  const float v_star = left ? -ust : ust;
  const float irs = __fdividef(1.0f, rs);
  const float tau = sub(irs, __fdividef(sub(ps, p_s), mul(W_s, W_s)));
  float rstar = (tau > 0.0f) ? __fdividef(1.0f, tau) : float(kRhoFloor);
  rstar = vmax(rstar, float(kRhoFloor));
  const float c_s = sqrtf(mul(mul(gs.gamma, p_s), irs));
  const float c_star = sqrtf(__fdividef(mul(gs.gamma, ps), rstar));
  const bool shock = ps > p_s;
  const float head = shock ? fma(W_s, irs, v_s) : add(v_s, c_s);
  const float tail = shock ? head : add(v_star, c_star);
  const bool orig = head <= 0.0f;
  const bool star = !orig && (tail > 0.0f);
  float r, u, p;
  if (orig) {
    r = rs; u = u_s; p = p_s;
  } else if (star) {
    r = rstar; u = ust; p = ps;
  } else {
    const float w = __fdividef(head, sub(head, tail));
    r = fma(w, sub(rstar, rs), rs);
    u = fma(w, sub(ust, u_s), u_s);
    p = fma(w, sub(ps, p_s), p_s);
  }
  float E;
  sampled_flux<NQ>(r, u, p, t, gs, F, E);
  if constexpr (NQ == 6) {
    F.c.y = mul(F.c.x, left ? Lc.c.y : Rc.c.y);
    *uf = u;
  }
}

// HLLC flux (ppm.cuh: hllc_flux, the same expressions), explicitly rounded.
template <int NQ>
__device__ __forceinline__ void hllc(const Cell<NQ>& Lc, const Cell<NQ>& Rc, const Gas<float>& gs, Cell<NQ>& F,
                                     float* uf) {
  const float rL = lo(Lc.c), uL = Lc.a.x, pL = Lc.a.y;
  const float rR = lo(Rc.c), uR = Rc.a.x, pR = Rc.a.y;
  const float cL = sqrtf(__fdividef(mul(gs.gamma, pL), rL));
  const float cR = sqrtf(__fdividef(mul(gs.gamma, pR), rR));
  const float SL = vmin(sub(uL, cL), sub(uR, cR));
  const float SR = vmax(add(uL, cL), add(uR, cR));
  const float mL = mul(rL, sub(SL, uL));
  const float mR = mul(rR, sub(SR, uR));
  const float Ss = __fdividef(add(sub(pR, pL), fma(mL, uL, -mul(mR, uR))), sub(mL, mR));
  const bool left = (SL >= 0.0f) || (Ss >= 0.0f);
  const float r = left ? rL : rR, u = left ? uL : uR, p = left ? pL : pR;
  const float2 t = left ? Lc.b : Rc.b;
  const float S = left ? SL : SR, m = left ? mL : mR;
  float E;
  sampled_flux<NQ>(r, u, p, t, gs, F, E);
  const bool outer = left ? (SL >= 0.0f) : !(SR > 0.0f);
  float e = 0.0f;
  if constexpr (NQ == 6) {
    e = left ? Lc.c.y : Rc.c.y;
    F.c.y = mul(F.c.x, e);
    *uf = outer ? u : Ss;
  }
  if (!outer) {   // F*_K = F_K + S_K (U*_K - U_K)
    const float fac = __fdividef(m, sub(S, Ss));
    const float2 S2 = splat<float2>(S);
    const float Us4 = mul(fac, fma(sub(Ss, u), add(Ss, __fdividef(p, m)), __fdividef(E, r)));
    F.a = fma(S2, sub(make_float2(mul(fac, Ss), Us4), make_float2(mul(r, u), E)), F.a);
    F.b = fma(S2, sub(mul(splat<float2>(fac), t), mul(splat<float2>(r), t)), F.b);
    if constexpr (NQ == 6)
      F.c = fma(S2, sub(make_float2(fac, mul(fac, e)), make_float2(r, mul(r, e))), F.c);
    else
      F.c = fma(S, sub(fac, r), F.c);
  }
}

// The interface flux of a method variant (RS & 1: HLLC, else two-shock).
template <int NQ, int RS>
__device__ __forceinline__ void flux(const Cell<NQ>& L, const Cell<NQ>& R, const Gas<float>& gs, Cell<NQ>& F,
                                     float* uf) {
  if (RS & 1) hllc<NQ>(L, R, gs, F, uf);
  else two_shock<NQ>(L, R, gs, F, uf);
}

// Sliding window of one pencil (see PencilWindow), fields in groups.
template <int NQ>
struct Window {
  Cell<NQ> w[5];    // primitives of cells k-4 .. k
  Cell<NQ> dm[2];   // slopes of cells k-2, k-1
  Cell<NQ> ai[3];   // interface values k-4+1/2 .. k-2+1/2
  Cell<NQ> wp;      // right-edge state of cell k-4
  Cell<NQ> fl;      // flux at interface k-5+1/2 (sweep-local order)
  float ft[3];      // shock detectors of cells k-4 .. k-2
  float eta[3];     // contact-steepening weights of cells k-4 .. k-2 (RS & 2)
  float dr[2];      // density slopes of cells k-4, k-3 (RS & 2)
  float ufl;        // interface velocity at k-5+1/2 (dual energy)
};

}  // namespace px
}  // namespace cello
