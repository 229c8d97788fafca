// Host-compiled entry points of the per-interface PPM arithmetic and its
// hand-written adjoint, and of the host operation count of a leaf's sweep,
// for CPU unit tests of the device math (the same CELLO_HD functions the
// kernels run).  Built into a separate test library; the product library
// does not contain it.
#include "adjoint.cuh"
#include "opcount.cu"

using namespace cello;

template <typename T>
static void flux_t(const double* U, double dtdx, double gamma, double* F) {
  T u[8][5], f[5];
  for (int c = 0; c < 8; ++c)
    for (int k = 0; k < 5; ++k) u[c][k] = T(U[c * 5 + k]);
  window_flux(u, T(dtdx), Gas<T>::make(gamma), f);
  for (int k = 0; k < 5; ++k) F[k] = double(f[k]);
}

template <typename T>
static void vjp_t(const double* U, double dtdx, double gamma, const double* Fb, double* Ub) {
  T u[8][5], fb[5], ub[8][5];
  for (int c = 0; c < 8; ++c)
    for (int k = 0; k < 5; ++k) {
      u[c][k] = T(U[c * 5 + k]);
      ub[c][k] = T(0);
    }
  for (int k = 0; k < 5; ++k) fb[k] = T(Fb[k]);
  window_flux_vjp(u, T(dtdx), Gas<T>::make(gamma), fb, ub);
  for (int c = 0; c < 8; ++c)
    for (int k = 0; k < 5; ++k) Ub[c * 5 + k] = double(ub[c][k]);
}

extern "C" {
void cello_hc_window_flux(const double* U, double dtdx, double gamma, int precision, double* F) {
  if (precision == 4) flux_t<float>(U, dtdx, gamma, F);
  else flux_t<double>(U, dtdx, gamma, F);
}
void cello_hc_window_flux_vjp(const double* U, double dtdx, double gamma, int precision, const double* Fb,
                              double* Ub) {
  if (precision == 4) vjp_t<float>(U, dtdx, gamma, Fb, Ub);
  else vjp_t<double>(U, dtdx, gamma, Fb, Ub);
}
// One leaf's sweep through the counting scalar (float32 arithmetic), its
// update written back into slab [fields][N^3]; counts[6] per phase.
void cello_hc_opcount_leaf(float* slab, int n, int g, int axis, int a0, int a1, int b0, int b1, double dtdx,
                           double gamma, int riemann, int steepen, int dual, unsigned long long* counts) {
  opcount_leaf(slab, n, g, axis, a0, a1, b0, b1, dtdx, gamma, riemann, steepen, dual, counts);
}
}
