// Algorithmic operation count of the directionally split PPM sweep
// (Sec. II.C): the sweep's own formulas (ppm.cuh) run on the host in float32
// arithmetic through a counting scalar type, over the same cell and
// interface ranges the sweep kernel covers.  The count is the numerator of
// the sweep kernel's ALU roofline: a property of the method on the given
// data (its branches follow the data), not of the compiled code.
//
// Counted as one operation each: add, subtract, multiply, divide, square
// root, comparison (so min / max through their comparison), absolute value
// and copysign.  Negation (an operand modifier on the GPU), selects,
// conversions, loads and stores are free.
#include "cello_internal.h"
#include "ppm.cuh"

#include <vector>

namespace cello {
namespace {

thread_local unsigned long long tl_ops = 0;

CELLO_HD void tick() {
#ifndef __CUDA_ARCH__
  ++tl_ops;
#endif
}

struct OpF {
  float v;
  OpF() = default;
  CELLO_HD constexpr OpF(float x) : v(x) {}
  CELLO_HD constexpr OpF(double x) : v(float(x)) {}
  CELLO_HD constexpr OpF(int x) : v(float(x)) {}
};

CELLO_HD OpF operator+(OpF a, OpF b) { tick(); return OpF(a.v + b.v); }
CELLO_HD OpF operator-(OpF a, OpF b) { tick(); return OpF(a.v - b.v); }
CELLO_HD OpF operator*(OpF a, OpF b) { tick(); return OpF(a.v * b.v); }
CELLO_HD OpF operator/(OpF a, OpF b) { tick(); return OpF(a.v / b.v); }
CELLO_HD OpF operator-(OpF a) { return OpF(-a.v); }
CELLO_HD bool operator<(OpF a, OpF b) { tick(); return a.v < b.v; }
CELLO_HD bool operator>(OpF a, OpF b) { tick(); return a.v > b.v; }
CELLO_HD bool operator<=(OpF a, OpF b) { tick(); return a.v <= b.v; }
CELLO_HD bool operator>=(OpF a, OpF b) { tick(); return a.v >= b.v; }
CELLO_HD bool operator==(OpF a, OpF b) { tick(); return a.v == b.v; }
CELLO_HD bool operator!=(OpF a, OpF b) { tick(); return a.v != b.v; }
// found by argument-dependent lookup from the templates of ppm.cuh
CELLO_HD OpF vabs(OpF a) { tick(); return OpF(fabsf(a.v)); }
CELLO_HD OpF vsqrt(OpF a) { tick(); return OpF(sqrtf(a.v)); }
CELLO_HD OpF vcopysign(OpF a, OpF b) { tick(); return OpF(copysignf(a.v, b.v)); }
CELLO_HD OpF vdiv(OpF a, OpF b) { tick(); return OpF(a.v / b.v); }

}  // namespace

// One leaf's pencils of one sweep, with the update written back (so that
// the next sweep of the step sees the swept state).  counts[6] receives the
// operations of the six phases of the kernel: primitives, slopes and shock
// detector, interface values, flattening + monotonicity + tracing, Riemann
// flux, conservative update.
void opcount_leaf(float* slab, int n, int g, int axis, int a0, int a1, int b0, int b1, double dtdx_d, double gamma,
                  int riemann, int steepen, unsigned long long counts[6]) {
  const int N = n + 2 * g;
  const long SLAB = (long)N * N * N;
  const long sAx = axis == 0 ? 1 : (axis == 1 ? N : (long)N * N);
  const long sTA = axis == 2 ? N : (long)N * N;
  const long sTB = axis == 0 ? N : 1;
  int comp[5];
  comp[0] = 0; comp[1] = 1 + axis; comp[4] = 4;
  comp[2] = axis == 0 ? 2 : 1;
  comp[3] = axis == 2 ? 2 : 3;
  const Gas<OpF> gs = Gas<OpF>::make(gamma);
  const OpF dtdx = OpF(dtdx_d);
  std::vector<OpF> Uc((size_t)N * 5), W((size_t)N * 5), dm((size_t)N * 5), ai((size_t)N * 5), Wm((size_t)N * 5),
      Wp((size_t)N * 5), F((size_t)N * 5), ft((size_t)N);
  auto mark = [&](int phase, unsigned long long before) { counts[phase] += tl_ops - before; };
  for (int pa = a0; pa < a1; ++pa)
    for (int pb = b0; pb < b1; ++pb) {
      float* base = slab + pa * sTA + pb * sTB;
      unsigned long long t0 = tl_ops;
      for (int j = 0; j < N; ++j) {
        OpF us[5], w[5];
        for (int f = 0; f < 5; ++f) Uc[j * 5 + f] = OpF(base[f * SLAB + j * sAx]);
        for (int k = 0; k < 5; ++k) us[k] = Uc[j * 5 + comp[k]];
        to_primitive(us, gs, w);
        for (int k = 0; k < 5; ++k) W[j * 5 + k] = w[k];
      }
      mark(0, t0);
      t0 = tl_ops;
      for (int j = 2; j <= N - 3; ++j) {
        for (int k = 0; k < 5; ++k)
          dm[j * 5 + k] = limited_slope(W[(j - 1) * 5 + k], W[j * 5 + k], W[(j + 1) * 5 + k]);
        ft[j] = flatten_tilde(W[(j - 2) * 5 + 4], W[(j - 1) * 5 + 4], W[(j + 1) * 5 + 4], W[(j + 2) * 5 + 4],
                              W[(j - 1) * 5 + 1], W[(j + 1) * 5 + 1]);
      }
      mark(1, t0);
      t0 = tl_ops;
      for (int j = 2; j <= N - 4; ++j)
        for (int k = 0; k < 5; ++k)
          ai[j * 5 + k] = interface_value(W[j * 5 + k], W[(j + 1) * 5 + k], dm[j * 5 + k], dm[(j + 1) * 5 + k]);
      mark(2, t0);
      t0 = tl_ops;
      for (int j = 3; j <= N - 4; ++j) {
        OpF sl = OpF(0), sr = OpF(0), e = OpF(0);
        if (steepen) {
          e = steepening_eta(W[(j - 2) * 5], W[(j - 1) * 5], W[j * 5], W[(j + 1) * 5], W[(j + 2) * 5],
                             W[(j - 1) * 5 + 4], W[(j + 1) * 5 + 4], gs.gamma);
          sl = W[(j - 1) * 5] + OpF(0.5) * dm[(j - 1) * 5];
          sr = W[(j + 1) * 5] - OpF(0.5) * dm[(j + 1) * 5];
        }
        const OpF s = W[(j + 1) * 5 + 4] - W[(j - 1) * 5 + 4];
        const OpF fj = ft[j], fm = ft[j - 1], fpp = ft[j + 1];
        const OpF f = (s > OpF(0)) ? vmax(fj, fm) : ((s < OpF(0)) ? vmax(fj, fpp) : fj);
        OpF w[5], aL[5], aR[5], m5[5], p5[5];
        for (int k = 0; k < 5; ++k) {
          w[k] = W[j * 5 + k];
          aL[k] = ai[(j - 1) * 5 + k];
          aR[k] = ai[j * 5 + k];
          if (steepen && k == 0) {
            aL[0] = aL[0] * (OpF(1) - e) + sl * e;
            aR[0] = aR[0] * (OpF(1) - e) + sr * e;
          }
          flatten_monotone(w[k], f, aL[k], aR[k]);
        }
        trace(w, aL, aR, dtdx, gs, m5, p5);
        for (int k = 0; k < 5; ++k) {
          Wm[j * 5 + k] = m5[k];
          Wp[j * 5 + k] = p5[k];
        }
      }
      mark(3, t0);
      t0 = tl_ops;
      for (int j = 3; j <= N - 5; ++j) {
        OpF L[5], R[5], fl[5];
        for (int k = 0; k < 5; ++k) {
          L[k] = Wp[j * 5 + k];
          R[k] = Wm[(j + 1) * 5 + k];
        }
        if (riemann == CELLO_RIEMANN_HLLC) hllc_flux(L, R, gs, fl);
        else riemann_flux(L, R, gs, fl);
        for (int k = 0; k < 5; ++k) F[j * 5 + k] = fl[k];
      }
      mark(4, t0);
      t0 = tl_ops;
      for (int j = g; j < g + n; ++j)
        for (int k = 0; k < 5; ++k) {
          const OpF v = Uc[j * 5 + comp[k]] - dtdx * (F[j * 5 + k] - F[(j - 1) * 5 + k]);
          base[comp[k] * SLAB + j * sAx] = v.v;
        }
      mark(5, t0);
    }
}

}  // namespace cello
