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
// flux, conservative update.  NQ = 6: the dual-energy formalism's sixth
// field (its passive reconstruction and flux, the compression term and the
// synchronisation in the update phase).
template <int NQ>
static void opcount_leaf_t(float* slab, int n, int g, int axis, int a0, int a1, int b0, int b1, double dtdx_d,
                           double gamma, int riemann, int steepen, unsigned long long counts[6]) {
  const int N = n + 2 * g;
  const long SLAB = (long)N * N * N;
  const long sAx = axis == 0 ? 1 : (axis == 1 ? N : (long)N * N);
  const long sTA = axis == 2 ? N : (long)N * N;
  const long sTB = axis == 0 ? N : 1;
  int comp[6];
  comp[0] = 0; comp[1] = 1 + axis; comp[4] = 4; comp[5] = 5;
  comp[2] = axis == 0 ? 2 : 1;
  comp[3] = axis == 2 ? 2 : 3;
  const Gas<OpF> gs = Gas<OpF>::make(gamma);
  const OpF dtdx = OpF(dtdx_d);
  const size_t NN = (size_t)N * NQ;
  std::vector<OpF> Uc(NN), W(NN), dm(NN), ai(NN), Wm(NN), Wp(NN), F(NN), ft((size_t)N), uf((size_t)N);
  auto mark = [&](int phase, unsigned long long before) { counts[phase] += tl_ops - before; };
  for (int pa = a0; pa < a1; ++pa)
    for (int pb = b0; pb < b1; ++pb) {
      float* base = slab + pa * sTA + pb * sTB;
      unsigned long long t0 = tl_ops;
      for (int j = 0; j < N; ++j) {
        OpF us[NQ], w[NQ];
        for (int f = 0; f < NQ; ++f) Uc[j * NQ + f] = OpF(base[f * SLAB + j * sAx]);
        for (int k = 0; k < NQ; ++k) us[k] = Uc[j * NQ + comp[k]];
        if constexpr (NQ == 6) to_primitive_de(us, gs, w);
        else to_primitive(us, gs, w);
        for (int k = 0; k < NQ; ++k) W[j * NQ + k] = w[k];
      }
      mark(0, t0);
      t0 = tl_ops;
      for (int j = 2; j <= N - 3; ++j) {
        for (int k = 0; k < NQ; ++k)
          dm[j * NQ + k] = limited_slope(W[(j - 1) * NQ + k], W[j * NQ + k], W[(j + 1) * NQ + k]);
        ft[j] = flatten_tilde(W[(j - 2) * NQ + 4], W[(j - 1) * NQ + 4], W[(j + 1) * NQ + 4], W[(j + 2) * NQ + 4],
                              W[(j - 1) * NQ + 1], W[(j + 1) * NQ + 1]);
      }
      mark(1, t0);
      t0 = tl_ops;
      for (int j = 2; j <= N - 4; ++j)
        for (int k = 0; k < NQ; ++k)
          ai[j * NQ + k] =
              interface_value(W[j * NQ + k], W[(j + 1) * NQ + k], dm[j * NQ + k], dm[(j + 1) * NQ + k]);
      mark(2, t0);
      t0 = tl_ops;
      for (int j = 3; j <= N - 4; ++j) {
        OpF sl = OpF(0), sr = OpF(0), e = OpF(0);
        if (steepen) {
          e = steepening_eta(W[(j - 2) * NQ], W[(j - 1) * NQ], W[j * NQ], W[(j + 1) * NQ], W[(j + 2) * NQ],
                             W[(j - 1) * NQ + 4], W[(j + 1) * NQ + 4], gs.gamma);
          sl = W[(j - 1) * NQ] + OpF(0.5) * dm[(j - 1) * NQ];
          sr = W[(j + 1) * NQ] - OpF(0.5) * dm[(j + 1) * NQ];
        }
        const OpF s = W[(j + 1) * NQ + 4] - W[(j - 1) * NQ + 4];
        const OpF fj = ft[j], fm = ft[j - 1], fpp = ft[j + 1];
        const OpF f = (s > OpF(0)) ? vmax(fj, fm) : ((s < OpF(0)) ? vmax(fj, fpp) : fj);
        OpF w[NQ], aL[NQ], aR[NQ], mq[NQ], pq[NQ];
        for (int k = 0; k < NQ; ++k) {
          w[k] = W[j * NQ + k];
          aL[k] = ai[(j - 1) * NQ + k];
          aR[k] = ai[j * NQ + k];
          if (steepen && k == 0) {
            aL[0] = aL[0] * (OpF(1) - e) + sl * e;
            aR[0] = aR[0] * (OpF(1) - e) + sr * e;
          }
          flatten_monotone(w[k], f, aL[k], aR[k]);
        }
        trace<OpF, NQ>(w, aL, aR, dtdx, gs, mq, pq);
        for (int k = 0; k < NQ; ++k) {
          Wm[j * NQ + k] = mq[k];
          Wp[j * NQ + k] = pq[k];
        }
      }
      mark(3, t0);
      t0 = tl_ops;
      for (int j = 3; j <= N - 5; ++j) {
        OpF L[NQ], R[NQ], fl[NQ];
        for (int k = 0; k < NQ; ++k) {
          L[k] = Wp[j * NQ + k];
          R[k] = Wm[(j + 1) * NQ + k];
        }
        OpF u = OpF(0);
        if (riemann == CELLO_RIEMANN_HLLC) hllc_flux<OpF, NQ>(L, R, gs, fl, &u);
        else riemann_flux<OpF, NQ>(L, R, gs, fl, &u);
        for (int k = 0; k < NQ; ++k) F[j * NQ + k] = fl[k];
        uf[j] = u;
      }
      mark(4, t0);
      t0 = tl_ops;
      for (int j = g; j < g + n; ++j) {
        OpF v[NQ];
        for (int k = 0; k < NQ; ++k) v[k] = Uc[j * NQ + comp[k]] - dtdx * (F[j * NQ + k] - F[(j - 1) * NQ + k]);
        if constexpr (NQ == 6) {
          v[5] = v[5] - (dtdx * W[j * NQ + 4]) * (uf[j] - uf[j - 1]);
          v[5] = dual_sync(v);
        }
        for (int k = 0; k < NQ; ++k) base[comp[k] * SLAB + j * sAx] = v[k].v;
      }
      mark(5, t0);
    }
}

void opcount_leaf(float* slab, int n, int g, int axis, int a0, int a1, int b0, int b1, double dtdx_d, double gamma,
                  int riemann, int steepen, int dual, unsigned long long counts[6]) {
  if (dual) opcount_leaf_t<6>(slab, n, g, axis, a0, a1, b0, b1, dtdx_d, gamma, riemann, steepen, counts);
  else opcount_leaf_t<5>(slab, n, g, axis, a0, a1, b0, b1, dtdx_d, gamma, riemann, steepen, counts);
}

}  // namespace cello
