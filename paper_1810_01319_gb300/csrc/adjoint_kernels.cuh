// Adjoint of one directional PPM sweep and of the periodic same-level ghost
// copy, with dt held fixed.  Included by the per-precision translation units.
#pragma once

#include "adjoint.cuh"
#include "cello_internal.h"

namespace cello {

// ---------------------------------------------------------------------
// Adjoint sweep.  The forward sweep maps U to U' with
//   U'_j = U_j - (dt/dx) (F_{j+1/2} - F_{j-1/2})  for updated cells j,
// F_{c+1/2} a function of cells c-3..c+4.  Given lam' (adjoint of U'), the
// adjoint of U is lam_j = lam'_j + sum_c (dF_c/dU_j)^T mu_c with
// mu_c = (dt/dx)(m_{c+1} lam'_{c+1} - m_c lam'_c), m = 1 on updated cells.
// One CTA item = P pencils; phase 1 stages U and lam', phase 2 computes
// each interface's vector-Jacobian product into shared memory, phase 3
// gathers the eight contributions of each cell in a fixed order.
// ---------------------------------------------------------------------
template <typename T, int NB, int P>
__global__ void __launch_bounds__((NB + 8) * P)
adjoint_sweep_kernel(DevMesh m, AdjSweepParams prm) {
  constexpr int G = kGhosts, N = NB + 2 * G, S = P + 1, A = N * S, NI = NB + 1;
  constexpr long SLAB = (long)N * N * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sU = reinterpret_cast<T*>(smem_raw);
  T* sL = sU + 5 * A;
  T* sC = sL + 5 * A;   // [NI][8][5][P]

  const Gas<T> gs = Gas<T>::make(m.gamma);
  const T* U = static_cast<const T*>(prm.U);
  T* lam = static_cast<T*>(prm.lam);
  const int axis = prm.axis;
  const int cA = prm.a1 - prm.a0, cB = prm.b1 - prm.b0;
  const long sAx = axis == 0 ? 1 : (axis == 1 ? N : (long)N * N);
  const long sTA = axis == 2 ? N : (long)N * N;
  const long sTB = axis == 0 ? N : 1;
  int comp[5];
  comp[0] = 0; comp[1] = 1 + axis; comp[4] = 4;
  comp[2] = axis == 0 ? 2 : 1;
  comp[3] = axis == 2 ? 2 : 3;
  const int t = threadIdx.x;
  const int lc = axis == 0 ? t % N : t / P;
  const int lp = axis == 0 ? t / N : t % P;
  __shared__ T s_dtdx[16];
  if (t <= m.max_level) s_dtdx[t] = T(*prm.dt / ldexp(m.dx0, -t));
  __syncthreads();

  for (int item = blockIdx.x; item < prm.n_items; item += gridDim.x) {
    const int leaf = prm.leaf0 + item / prm.tiles_per_leaf;
    const int tile = item % prm.tiles_per_leaf;
    const T dtdx = s_dtdx[m.leaf[leaf].x];
    const int q = tile * P + lp;
    const bool valid = q < cA * cB;
    const int pa = prm.a0 + (valid ? q / cB : 0), pb = prm.b0 + (valid ? q % cB : 0);
    const long off = (long)leaf * 5 * SLAB + pa * sTA + pb * sTB + lc * sAx;
    if (valid) {
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        sU[k * A + lc * S + lp] = U[off + comp[k] * SLAB];
        sL[k * A + lc * S + lp] = lam[off + comp[k] * SLAB];
      }
    }
    __syncthreads();
    if (t < NI * P) {
      const int p = t % P, ci = t / P, c = 3 + ci;
      const T m0 = (c >= G && c < G + NB) ? T(1) : T(0);
      const T m1 = (c + 1 >= G && c + 1 < G + NB) ? T(1) : T(0);
      T mu[5];
      bool any = false;
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        mu[k] = dtdx * (m1 * sL[k * A + (c + 1) * S + p] - m0 * sL[k * A + c * S + p]);
        any = any || (mu[k] != T(0));
      }
      T Ub[8][5];
#pragma unroll
      for (int c8 = 0; c8 < 8; ++c8)
#pragma unroll
        for (int k = 0; k < 5; ++k) Ub[c8][k] = T(0);
      if (any) {
        T W8[8][5];
#pragma unroll
        for (int c8 = 0; c8 < 8; ++c8)
#pragma unroll
          for (int k = 0; k < 5; ++k) W8[c8][k] = sU[k * A + (c - 3 + c8) * S + p];
        window_flux_vjp(W8, dtdx, gs, mu, Ub);
      }
#pragma unroll
      for (int c8 = 0; c8 < 8; ++c8)
#pragma unroll
        for (int k = 0; k < 5; ++k) sC[((ci * 8 + c8) * 5 + k) * P + p] = Ub[c8][k];
    }
    __syncthreads();
    if (valid) {
      const int ci0 = lc - 7 > 0 ? lc - 7 : 0;
      const int ci1 = lc < NI - 1 ? lc : NI - 1;
#pragma unroll
      for (int k = 0; k < 5; ++k) {
        T v = sL[k * A + lc * S + lp];
        for (int ci = ci0; ci <= ci1; ++ci) v += sC[((ci * 8 + (lc - ci)) * 5 + k) * P + lp];
        lam[off + comp[k] * SLAB] = v;
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------
// Transposed periodic same-level ghost copy: every interior cell gathers the
// adjoints of the ghost cells copied from it (directions in table order),
// then all ghost adjoints are cleared.
// ---------------------------------------------------------------------
template <typename T, int NB>
__global__ void __launch_bounds__(256) adjoint_refresh_gather_kernel(DevMesh m, T* lam) {
  constexpr int G = kGhosts, N = NB + 2 * G;
  constexpr long SLAB = (long)N * N * N;
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long)m.B * NB * NB * NB) return;
  const int leaf = (int)(gid / (NB * NB * NB));
  const int i = (int)(gid % (NB * NB * NB));
  const int s[3] = {i % NB + G, (i / NB) % NB + G, i / (NB * NB) + G};
  T acc[5];
  const long own = (long)leaf * 5 * SLAB + ((long)s[2] * N + s[1]) * N + s[0];
#pragma unroll
  for (int f = 0; f < 5; ++f) acc[f] = lam[own + f * SLAB];
  for (int e = 0; e < 27; ++e) {
    if (e == 13) continue;
    const int d[3] = {e % 3 - 1, (e / 3) % 3 - 1, e / 9 - 1};
    int c[3];
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      c[a] = s[a] + d[a] * NB;
      ok = ok && c[a] >= 0 && c[a] < N;
    }
    if (!ok) continue;
    const int back = (-d[2] + 1) * 9 + (-d[1] + 1) * 3 + (-d[0] + 1);
    const int src = m.idx[leaf * 27 + back];   // the leaf whose ghost in direction d copies this cell
    const long o = (long)src * 5 * SLAB + ((long)c[2] * N + c[1]) * N + c[0];
#pragma unroll
    for (int f = 0; f < 5; ++f) acc[f] += lam[o + f * SLAB];
  }
#pragma unroll
  for (int f = 0; f < 5; ++f) lam[own + f * SLAB] = acc[f];
}

template <typename T, int NB>
__global__ void __launch_bounds__(256) zero_ghosts_kernel(T* lam, int B) {
  constexpr int G = kGhosts, N = NB + 2 * G, NG = N * N * N - NB * NB * NB;
  constexpr long SLAB = (long)N * N * N;
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long)B * NG) return;
  const int leaf = (int)(gid / NG);
  int x, y, z;
  ghost_coord<NB>((int)(gid % NG), x, y, z);
  const long o = (long)leaf * 5 * SLAB + ((long)z * N + y) * N + x;
#pragma unroll
  for (int f = 0; f < 5; ++f) lam[o + f * SLAB] = T(0);
}

}  // namespace cello
