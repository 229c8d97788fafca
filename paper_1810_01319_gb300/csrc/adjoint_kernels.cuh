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
      for (int k = 0; k < 5; ++k) mu[k] = dtdx * (m1 * sL[k * A + (c + 1) * S + p] - m0 * sL[k * A + c * S + p]);
      if (prm.regb && (c == G - 1 || c == G + NB - 1)) {   // flux kept for the coarse-fine correction
        const int qq = tile * P + p;
        if (qq < cA * cB) {
          const int ca = prm.a0 + qq / cB, cb = prm.b0 + qq % cB;
          if (ca >= G && ca < G + NB && cb >= G && cb < G + NB) {
            const int slot = m.face_slot[leaf * 6 + 2 * axis + (c == G - 1 ? 0 : 1)];
            if (slot >= 0) {
              const double* r = prm.regb + (long)slot * 5 * NB * NB + (ca - G) * NB + (cb - G);
#pragma unroll
              for (int k = 0; k < 5; ++k) mu[k] += T(r[(long)comp[k] * NB * NB]);
            }
          }
        }
      }
#pragma unroll
      for (int k = 0; k < 5; ++k) any = any || (mu[k] != T(0));
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

// ---------------------------------------------------------------------
// AMR transpose of the ghost refresh.  Each ghost cell's adjoint is added to
// the cells its forward value was made from, with the forward's weights:
// copy 1; restriction 0.125 on each of 8 cells; prolongation U_C + 0.25
// sum_d s_d D_d with D_d = minmod(U_C - U_m, U_p - U_C) differentiated along
// the branch the forward took (per field), the neighbour values U_m, U_p
// being copies, restrictions or injections of further cells.  Sources are
// leaf interiors, ghosts are only read, so atomic adds suffice.
// ---------------------------------------------------------------------
template <typename T, int NB>
__device__ __forceinline__ void add5(T* lam, int leaf, int x, int y, int z, const T w[5]) {
  constexpr int N = NB + 2 * kGhosts;
  constexpr long SLAB = (long)N * N * N;
  T* b = lam + (long)leaf * 5 * SLAB + ((long)z * N + y) * N + x;
#pragma unroll
  for (int f = 0; f < 5; ++f)
    if (w[f] != T(0)) atomicAdd(b + f * SLAB, w[f]);
}

template <typename T, int NB>
__device__ __forceinline__ void add_restrict8(T* lam, int leaf, int fx, int fy, int fz, const T w[5]) {
  T w8[5];
#pragma unroll
  for (int f = 0; f < 5; ++f) w8[f] = w[f] * T(0.125);
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) add5<T, NB>(lam, leaf, fx + dx, fy + dy, fz + dz, w8);
}

// Adjoint of slope_neighbour: w onto the sources of that neighbour value.
template <typename T, int NB>
__device__ void slope_neighbour_bwd(const DevMesh& m, T* lam, int C, const int rc[3], int a, int side, const T w[5]) {
  constexpr int G = kGhosts, H = NB / 2;
  const int e = C * 27 + face_dir(a, side);
  const int8_t k = m.kind[e];
  if (k == kBoundary) {
    add5<T, NB>(lam, C, rc[0] + G, rc[1] + G, rc[2] + G, w);
    return;
  }
  int r2[3] = {rc[0], rc[1], rc[2]};
  r2[a] = side < 0 ? NB - 1 : 0;
  if (k == kSame) {
    add5<T, NB>(lam, m.idx[e], r2[0] + G, r2[1] + G, r2[2] + G, w);
  } else if (k == kFine) {
    const int o0 = r2[0] / H, o1 = r2[1] / H, o2 = r2[2] / H;
    const int child = m.fine8[e * 8 + o2 * 4 + o1 * 2 + o0];
    add_restrict8<T, NB>(lam, child, 2 * r2[0] - o0 * NB + G, 2 * r2[1] - o1 * NB + G, 2 * r2[2] - o2 * NB + G, w);
  } else {
    const int4 cl = m.leaf[C];
    const int K = m.idx[e];
    const int4 kl = m.leaf[K];
    int g[3] = {cl.y * NB + rc[0], cl.z * NB + rc[1], cl.w * NB + rc[2]};
    g[a] += side;
    g[a] = wrap_mod(g[a], (m.root[a] << cl.x) * NB);
    add5<T, NB>(lam, K, (g[0] >> 1) - kl.y * NB + G, (g[1] >> 1) - kl.z * NB + G, (g[2] >> 1) - kl.w * NB + G, w);
  }
}

template <typename T, int NB>
__global__ void __launch_bounds__(256) adjoint_refresh_scatter_kernel(DevMesh m, const T* U, T* lam) {
  constexpr int G = kGhosts, N = NB + 2 * G, NG = N * N * N - NB * NB * NB, H = NB / 2;
  constexpr long SLAB = (long)N * N * N;
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long)m.B * NG) return;
  const int leaf = (int)(gid / NG);
  int c[3];
  ghost_coord<NB>((int)(gid % NG), c[0], c[1], c[2]);
  const long own = (long)leaf * 5 * SLAB + ((long)c[2] * N + c[1]) * N + c[0];
  T lg[5];
  bool any = false;
#pragma unroll
  for (int f = 0; f < 5; ++f) {
    lg[f] = lam[own + f * SLAB];
    any = any || lg[f] != T(0);
  }
  if (!any) return;
  int d[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    d[a] = c[a] < G ? -1 : (c[a] >= G + NB ? 1 : 0);
    if (d[a] != 0 && m.kind[leaf * 27 + face_dir(a, d[a])] == kBoundary) {
      c[a] = d[a] < 0 ? G : G + NB - 1;
      d[a] = 0;
    }
  }
  const int e = leaf * 27 + (d[2] + 1) * 9 + (d[1] + 1) * 3 + (d[0] + 1);
  const int8_t k = m.kind[e];
  if (k == kSame) {
    add5<T, NB>(lam, m.idx[e], c[0] - d[0] * NB, c[1] - d[1] * NB, c[2] - d[2] * NB, lg);
    return;
  }
  if (k == kFine) {
    int r[3], o[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      r[a] = c[a] - G - d[a] * NB;
      o[a] = r[a] / H;
    }
    const int child = m.fine8[e * 8 + o[2] * 4 + o[1] * 2 + o[0]];
    add_restrict8<T, NB>(lam, child, 2 * r[0] - o[0] * NB + G, 2 * r[1] - o[1] * NB + G, 2 * r[2] - o[2] * NB + G, lg);
    return;
  }
  // prolongation from the coarser leaf C, differentiated along the forward's branches
  const int4 lf = m.leaf[leaf];
  const int C = m.idx[e];
  const int4 cl = m.leaf[C];
  const int L = lf.x;
  const int lij[3] = {lf.y, lf.z, lf.w}, cij[3] = {cl.y, cl.z, cl.w};
  int rc[3];
  T sgn[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int ncell = (m.root[a] << L) * NB;
    const int gl = wrap_mod(lij[a] * NB + (c[a] - G), ncell);
    rc[a] = (gl >> 1) - cij[a] * NB;
    sgn[a] = (gl & 1) ? T(1) : T(-1);
  }
  T Uc[5];
  load5<T, NB>(U, C, rc[0] + G, rc[1] + G, rc[2] + G, Uc);
  T wc[5];
#pragma unroll
  for (int f = 0; f < 5; ++f) wc[f] = lg[f];
  for (int a = 0; a < 3; ++a) {
    T Um[5], Up[5];
    int rm[3] = {rc[0], rc[1], rc[2]}, rp[3] = {rc[0], rc[1], rc[2]};
    rm[a] -= 1;
    rp[a] += 1;
    if (rm[a] >= 0) load5<T, NB>(U, C, rm[0] + G, rm[1] + G, rm[2] + G, Um);
    else slope_neighbour<T, NB>(m, U, C, rc, a, -1, Uc, Um);
    if (rp[a] < NB) load5<T, NB>(U, C, rp[0] + G, rp[1] + G, rp[2] + G, Up);
    else slope_neighbour<T, NB>(m, U, C, rc, a, 1, Uc, Up);
    T wm[5], wp[5];
#pragma unroll
    for (int f = 0; f < 5; ++f) {
      const T lo = Uc[f] - Um[f], hi = Up[f] - Uc[f];
      const T gD = T(0.25) * sgn[a] * lg[f];   // adjoint of D_a
      wm[f] = T(0);
      wp[f] = T(0);
      if (lo * hi > T(0)) {
        if (vabs(lo) <= vabs(hi)) {   // D = U_C - U_m
          wc[f] += gD;
          wm[f] = -gD;
        } else {                      // D = U_p - U_C
          wc[f] -= gD;
          wp[f] = gD;
        }
      }
    }
    if (rm[a] >= 0) add5<T, NB>(lam, C, rm[0] + G, rm[1] + G, rm[2] + G, wm);
    else slope_neighbour_bwd<T, NB>(m, lam, C, rc, a, -1, wm);
    if (rp[a] < NB) add5<T, NB>(lam, C, rp[0] + G, rp[1] + G, rp[2] + G, wp);
    else slope_neighbour_bwd<T, NB>(m, lam, C, rc, a, 1, wp);
  }
  add5<T, NB>(lam, C, rc[0] + G, rc[1] + G, rc[2] + G, wc);
}

// Adjoint of the coarse-fine flux correction: with lam the adjoint after the
// step, d/dF_c = s (dt/dx_c) lam_c and each of the four fine fluxes gets
// -0.25 s (dt/dx_c) lam_c.  One thread per coarse face cell.
template <typename T, int NB>
__global__ void __launch_bounds__(256) fluxcorr_adjoint_kernel(DevMesh m, const T* lam, const CoarseFace* faces,
                                                               int nfaces, double* regb, const double* dt) {
  constexpr int G = kGhosts, N = NB + 2 * G, H = NB / 2;
  constexpr long SLAB = (long)N * N * N;
  constexpr long FS = (long)NB * NB;
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long)nfaces * NB * NB) return;
  const CoarseFace cf = faces[gid / (NB * NB)];
  const int i = (int)(gid % (NB * NB));
  const int t1 = i % NB, t2 = i / NB;
  const int4 cl = m.leaf[cf.leaf];
  const double coef = (*dt / ldexp(m.dx0, -cl.x)) * double(cf.side);
  const int t1a = cf.axis == 0 ? 1 : 0, t2a = cf.axis == 2 ? 1 : 2;
  int cc[3];
  cc[cf.axis] = cf.side > 0 ? G + NB - 1 : G;
  cc[t1a] = G + t1;
  cc[t2a] = G + t2;
  const T* cell = lam + (long)cf.leaf * 5 * SLAB + ((long)cc[2] * N + cc[1]) * N + cc[0];
  const int o1 = t1 / H, o2 = t2 / H, b1 = t1 - o1 * H, b2 = t2 - o2 * H;
  double* Rc = regb + (long)cf.cslot * 5 * FS + t2 * NB + t1;
  double* Rf = regb + (long)cf.fslot[o2 * 2 + o1] * 5 * FS + (2 * b2) * NB + 2 * b1;
#pragma unroll
  for (int f = 0; f < 5; ++f) {
    const double g = coef * double(cell[f * SLAB]);
    Rc[f * FS] = g;
    const double gf = -0.25 * g;
    double* r = Rf + f * FS;
    r[0] = gf;
    r[1] = gf;
    r[NB] = gf;
    r[NB + 1] = gf;
  }
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
