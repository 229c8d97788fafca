// Templated kernels of the hydro step.  Included by the per-precision
// translation units, which fix the FMA policy (float64: no contraction).
#pragma once

#include "cello_internal.h"
#include "ppm.cuh"
#include "stream_x2.cuh"

namespace cello {

__device__ __forceinline__ int wrap_mod(int v, int m) {
  int r = v % m;
  return r < 0 ? r + m : r;
}

template <typename T>
__device__ __forceinline__ T minmod(T a, T b) {
  return (a * b > T(0)) ? ((vabs(a) <= vabs(b)) ? a : b) : T(0);
}

// =====================================================================
// Directional PPM sweep.  One CTA item = P pencils of one leaf; a thread
// owns one cell of one pencil (pencil index fastest across the threads of a
// warp).  Shared arrays are [NQ][N][P], pencil fastest, so that a warp's
// accesses at one stencil offset fall in consecutive banks.  Phases:
//   1 load + primitives  2 limited slopes, shock detector  3 interface
//   values  4 flatten + monotone + trace  5 Riemann flux (+ face registers)
//   6 conservative update of cells g..g+n-1.
// =====================================================================
// The method variant of a sweep kernel, fixed at compile time so that each
// kernel carries only what it uses: RS = solver | 2 * steepening | 4 * dual
// energy, solver CELLO_RIEMANN_TWO_SHOCK (0) or CELLO_RIEMANN_HLLC (1),
// steepening and dual energy 0 or 1.
__host__ __device__ constexpr int method_code(int riemann, int steepen, int dual = 0) {
  return riemann | (steepen << 1) | (dual << 2);
}

// Shared arrays of N x P values of the shared-memory sweep: four groups of
// one per primitive (5, or 6 with dual energy), the shock detector, three
// for contact steepening, one for the interface velocities of dual energy.
__host__ __device__ constexpr int sweep_arrays(int RS) {
  return 4 * ((RS & 4) ? 6 : 5) + 1 + ((RS & 2) ? 3 : 0) + ((RS & 4) ? 1 : 0);
}

template <int RS, typename T>
__device__ __forceinline__ void interface_flux(const T L[5], const T R[5], const Gas<T>& gs, T F[5]) {
  if (RS & 1) hllc_flux(L, R, gs, F);
  else riemann_flux_bulk(L, R, gs, F);
}

template <int RS, typename T>
__device__ __forceinline__ void interface_flux6(const T L[6], const T R[6], const Gas<T>& gs, T F[6], T* uf) {
  if (RS & 1) hllc_flux<T, 6>(L, R, gs, F, uf);
  else riemann_flux_bulk6(L, R, gs, F, uf);
}

template <typename T, int NB, int P, int MINB, int RS>
__global__ void __launch_bounds__((NB + 8) * P, MINB)
sweep_kernel(DevMesh m, SweepParams prm) {
  constexpr int G = kGhosts, N = NB + 2 * G, S = P, A = N * S;
  constexpr long SLAB = (long)N * N * N;
  constexpr bool DE = (RS & 4) != 0;   // dual energy: a sixth field rho e
  constexpr int NQ = DE ? 6 : 5;
  // float32 evaluates the per-field formulas as the streaming form does
  // (stream_x2.cuh), so the two forms round alike
  constexpr bool kPacked = std::is_same<T, float>::value;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sW = reinterpret_cast<T*>(smem_raw);
  T* sA = sW + NQ * A;  // slopes, then left-edge states
  T* sB = sA + NQ * A;  // interface values, then fluxes
  T* sC = sB + NQ * A;  // right-edge states
  T* sFT = sC + NQ * A; // shock detector
  T* sE = sFT + A;      // contact-steepening weight (RS & 2 only)
  T* sDL = sE + A;      // density left-edge value of the steepened profile
  T* sDR = sDL + A;     // density right-edge value of the steepened profile
  T* sUF = sFT + A + ((RS & 2) ? 3 * A : 0);   // interface velocities (dual energy only)

  const Gas<T> gs = Gas<T>::make(m.gamma);
  T* U = static_cast<T*>(prm.U);
  const int axis = prm.axis;
  const int cA = prm.a1 - prm.a0, cB = prm.b1 - prm.b0;
  const long sAx = axis == 0 ? 1 : (axis == 1 ? N : (long)N * N);
  const long sTA = axis == 2 ? N : (long)N * N;   // transverse A: z (x, y sweeps) or y (z sweep)
  const long sTB = axis == 0 ? N : 1;             // transverse B: y (x sweep) or x (y, z sweeps)
  int comp[6];
  comp[0] = 0; comp[1] = 1 + axis; comp[4] = 4; comp[5] = 5;
  comp[2] = axis == 0 ? 2 : 1;
  comp[3] = axis == 2 ? 2 : 3;

  const int t = threadIdx.x;
  const int lc = t / P, lp = t % P;           // this thread's cell and pencil
  const int cp = lp, cj = lc;
  __shared__ int s_item;
  __shared__ T s_dtdx[16];
  // dt/dx per level, once per CTA (a float64 division per thread and item
  // would occupy the GPU's slow float64 pipe)
  if (t <= m.max_level) s_dtdx[t] = T(*prm.dt / ldexp(m.dx0, -t));
  __syncthreads();

  int item = blockIdx.x;
  if (prm.work) {
    if (t == 0) s_item = (int)atomicAdd(prm.work, 1u);
    __syncthreads();
    item = s_item;
  }
  while (item < prm.n_items) {
    const int lrel = (int)prm.div_tiles.div((unsigned)item);
    const int leaf = prm.leaf0 + lrel;
    const int tile = item - lrel * prm.tiles_per_leaf;
    const int4 lf = m.leaf[leaf];
    const T dtdx = s_dtdx[lf.x];

    // ---- phase 1
    const int q = tile * P + lp;
    const bool valid = q < cA * cB;
    const int qa = (int)prm.div_cb.div((unsigned)q);
    const int pa = prm.a0 + (valid ? qa : 0), pb = prm.b0 + (valid ? q - qa * cB : 0);
    T* base = U + (long)leaf * NQ * SLAB + pa * sTA + pb * sTB + lc * sAx;
    T Uc[NQ];
    if (valid) {
#pragma unroll
      for (int f = 0; f < NQ; ++f) Uc[f] = base[f * SLAB];
      T Us[NQ], W[NQ];
#pragma unroll
      for (int k = 0; k < NQ; ++k) Us[k] = Uc[comp[k]];
      if constexpr (kPacked) {
        const px::Cell<NQ> Wc = px::primitives<NQ>(Us, gs);
#pragma unroll
        for (int k = 0; k < NQ; ++k) W[k] = Wc.get(k);
      } else if constexpr (DE) {
        to_primitive_de(Us, gs, W);
      } else {
        to_primitive(Us, gs, W);
      }
#pragma unroll
      for (int k = 0; k < NQ; ++k) sW[k * A + lc * S + lp] = W[k];
    }
    __syncthreads();

    const int j = cj, p = cp;
    // ---- phase 2 (slopes of cells 2..N-3: the interfaces used below are 2..N-4)
    if (j >= 2 && j <= N - 3) {
#pragma unroll
      for (int k = 0; k < NQ; ++k) {
        const T* a = sW + k * A + p;
        if constexpr (kPacked) sA[k * A + j * S + p] = px::slope(a[(j - 1) * S], a[j * S], a[(j + 1) * S]);
        else sA[k * A + j * S + p] = limited_slope(a[(j - 1) * S], a[j * S], a[(j + 1) * S]);
      }
    }
    if (j >= 2 && j <= N - 3) {
      const T* pr = sW + 4 * A + p;
      const T* un = sW + 1 * A + p;
      sFT[j * S + p] = flatten_tilde(pr[(j - 2) * S], pr[(j - 1) * S], pr[(j + 1) * S], pr[(j + 2) * S],
                                     un[(j - 1) * S], un[(j + 1) * S]);
    }
    __syncthreads();
    // ---- phase 3 (interfaces j+1/2 read by cells 3..N-4)
    if (j >= 2 && j <= N - 4) {
#pragma unroll
      for (int k = 0; k < NQ; ++k) {
        if constexpr (kPacked)
          sB[k * A + j * S + p] = px::interface_val(sW[k * A + j * S + p], sW[k * A + (j + 1) * S + p],
                                                    sA[k * A + j * S + p], sA[k * A + (j + 1) * S + p]);
        else
          sB[k * A + j * S + p] = interface_value(sW[k * A + j * S + p], sW[k * A + (j + 1) * S + p],
                                                  sA[k * A + j * S + p], sA[k * A + (j + 1) * S + p]);
      }
    }
    if ((RS & 2) && j >= 3 && j <= N - 4) {   // contact steepening of cell j (density)
      const T* r = sW + p;
      const T* pr = sW + 4 * A + p;
      if constexpr (kPacked)
        sE[j * S + p] = px::steepening(r[(j - 2) * S], r[(j - 1) * S], r[j * S], r[(j + 1) * S], r[(j + 2) * S],
                                       pr[(j - 1) * S], pr[(j + 1) * S], gs.gamma);
      else
        sE[j * S + p] = steepening_eta(r[(j - 2) * S], r[(j - 1) * S], r[j * S], r[(j + 1) * S], r[(j + 2) * S],
                                       pr[(j - 1) * S], pr[(j + 1) * S], gs.gamma);
      sDL[j * S + p] = r[(j - 1) * S] + T(0.5) * sA[(j - 1) * S + p];
      sDR[j * S + p] = r[(j + 1) * S] - T(0.5) * sA[(j + 1) * S + p];
    }
    __syncthreads();
    // ---- phase 4
    if (j >= 3 && j <= N - 4) {
      const T* pr = sW + 4 * A + p;
      const T s = pr[(j + 1) * S] - pr[(j - 1) * S];
      const T fj = sFT[j * S + p], fm = sFT[(j - 1) * S + p], fpp = sFT[(j + 1) * S + p];
      const T f = (s > T(0)) ? vmax(fj, fm) : ((s < T(0)) ? vmax(fj, fpp) : fj);
      T W[NQ], aL[NQ], aR[NQ], Wm[NQ], Wp[NQ];
#pragma unroll
      for (int k = 0; k < NQ; ++k) {
        W[k] = sW[k * A + j * S + p];
        aL[k] = sB[k * A + (j - 1) * S + p];
        aR[k] = sB[k * A + j * S + p];
        if ((RS & 2) && k == 0) {
          const T e = sE[j * S + p];
          if constexpr (kPacked) {
            const float ome = px::sub(1.0f, e);
            aL[0] = px::fma(aL[0], ome, px::mul(sDL[j * S + p], e));
            aR[0] = px::fma(aR[0], ome, px::mul(sDR[j * S + p], e));
          } else {
            aL[0] = aL[0] * (T(1) - e) + sDL[j * S + p] * e;
            aR[0] = aR[0] * (T(1) - e) + sDR[j * S + p] * e;
          }
        }
        if constexpr (kPacked) px::flatten_mono(W[k], f, px::sub(1.0f, f), aL[k], aR[k]);
        else flatten_monotone(W[k], f, aL[k], aR[k]);
      }
      if constexpr (kPacked) {
        px::Cell<NQ> Wc, aLc, aRc, Wmc, Wpc;
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
          Wc.set(k, W[k]);
          aLc.set(k, aL[k]);
          aRc.set(k, aR[k]);
        }
        px::trace_cell<NQ>(Wc, aLc, aRc, px::splat<float2>(dtdx), gs, Wmc, Wpc);
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
          Wm[k] = Wmc.get(k);
          Wp[k] = Wpc.get(k);
        }
      } else {
        trace<T, NQ>(W, aL, aR, dtdx, gs, Wm, Wp);
      }
#pragma unroll
      for (int k = 0; k < NQ; ++k) {
        sA[k * A + j * S + p] = Wm[k];
        sC[k * A + j * S + p] = Wp[k];
      }
    }
    __syncthreads();
    // ---- phase 5
    if (j >= 3 && j <= N - 5) {
      T L[NQ], R[NQ], F[NQ];
#pragma unroll
      for (int k = 0; k < NQ; ++k) {
        L[k] = sC[k * A + j * S + p];
        R[k] = sA[k * A + (j + 1) * S + p];
      }
      if constexpr (kPacked) {
        px::Cell<NQ> Lc, Rc, Fc;
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
          Lc.set(k, L[k]);
          Rc.set(k, R[k]);
        }
        float uf = 0.0f;
        px::flux<NQ, RS>(Lc, Rc, gs, Fc, &uf);
#pragma unroll
        for (int k = 0; k < NQ; ++k) F[k] = Fc.get(k);
        if constexpr (DE) sUF[j * S + p] = uf;
      } else if constexpr (DE) {
        T uf;
        interface_flux6<RS>(L, R, gs, F, &uf);
        sUF[j * S + p] = uf;
      } else {
        interface_flux<RS>(L, R, gs, F);
      }
#pragma unroll
      for (int k = 0; k < NQ; ++k) sB[k * A + j * S + p] = F[k];
      if (prm.reg && (j == G - 1 || j == G + NB - 1)) {
        const int qq = tile * P + p;
        if (qq < cA * cB) {
          const int qqa = (int)prm.div_cb.div((unsigned)qq);
          const int ca = prm.a0 + qqa, cb = prm.b0 + qq - qqa * cB;
          if (ca >= G && ca < G + NB && cb >= G && cb < G + NB) {
            const int face = 2 * axis + (j == G - 1 ? 0 : 1);
            const int slot = m.face_slot[leaf * 6 + face];
            if (slot >= 0) {
              double* r = prm.reg + (long)slot * NQ * NB * NB + (ca - G) * NB + (cb - G);
#pragma unroll
              for (int k = 0; k < NQ; ++k) r[(long)comp[k] * NB * NB] = double(F[k]);
            }
          }
        }
      }
    }
    __syncthreads();
    // ---- phase 6 (dual energy: rho e also takes the compression term
    // -(dt/dx) p (u+ - u-) with the cell's pressure, then the synchronisation)
    if (valid && lc >= G && lc < G + NB) {
      T Un[NQ];
#pragma unroll
      for (int k = 0; k < NQ; ++k) {
        const T Fp = sB[k * A + lc * S + lp], Fm = sB[k * A + (lc - 1) * S + lp];
        if constexpr (kPacked) Un[k] = px::fma(-dtdx, px::sub(Fp, Fm), Uc[comp[k]]);
        else Un[k] = Uc[comp[k]] - dtdx * sub_rn(Fp, Fm);
      }
      if constexpr (DE) {
        const T pc = sW[4 * A + lc * S + lp];
        if constexpr (kPacked)
          Un[5] = px::fma(-px::mul(dtdx, pc), px::sub(sUF[lc * S + lp], sUF[(lc - 1) * S + lp]), Un[5]);
        else
          Un[5] = Un[5] - (dtdx * pc) * sub_rn(sUF[lc * S + lp], sUF[(lc - 1) * S + lp]);
        if constexpr (kPacked) Un[5] = px::dual_sync6(Un);
        else Un[5] = dual_sync(Un);
      }
#pragma unroll
      for (int k = 0; k < NQ; ++k) base[comp[k] * SLAB] = Un[k];
    }
    __syncthreads();
    if (prm.work) {
      if (t == 0) s_item = (int)atomicAdd(prm.work, 1u);
      __syncthreads();
      item = s_item;
    } else {
      item += gridDim.x;
    }
  }
}

// =====================================================================
// Register-streaming form of the same sweep: one thread per pencil walks
// its cells once, keeping a sliding window of the pencil in registers
// (primitives of 5 cells, 2 slopes, 3 shock detectors, 3 interface values,
// the last right-edge state and the last flux, each of 5 fields or 6 with
// dual energy), so that no value passes
// through shared memory and no phase waits at a barrier.  At step k the
// thread reads cell k and produces: the slope of cell k-1, the shock
// detector of cell k-2, the interface value k-2+1/2, the traced edge states
// of cell k-3, the flux at interface k-4+1/2 and the updated cell k-4.  The
// index ranges of every quantity are those of sweep_kernel, so the two
// forms evaluate the same expressions on the same values.
// =====================================================================
// The sliding window of one pencil.
// NQ = 6 with the dual-energy formalism (e as a sixth primitive).
template <typename T, int NQ = 5>
struct PencilWindow {
  T w[5][NQ];   // primitives of cells k-4 .. k (sweep-local components)
  T dm[2][NQ];  // slopes of cells k-2, k-1
  T ft[3];      // shock detectors of cells k-4 .. k-2
  T ai[3][NQ];  // interface values k-4+1/2 .. k-2+1/2
  T wp[NQ];     // right-edge state of cell k-4 (left state of interface k-4+1/2)
  T fl[NQ];     // flux at interface k-5+1/2
  T eta[3];     // contact-steepening weights of cells k-4 .. k-2 (RS & 2)
  T dr[2];      // density slopes of cells k-4, k-3 (RS & 2)
  T ufl;        // interface-state velocity at k-5+1/2 (dual energy)
};

// One step of the walk: cell k enters as conserved values Us (sweep-local
// components); old holds cell k-4 as stored (component order), read
// before it is overwritten here.
// DEFER: the updated cell is returned in upd[NQ] (component order) instead
// of being stored.  RS & 4 (dual energy): six fields, rho e taking the
// compression term with the pressure of its cell and the synchronisation.
template <typename T, int NB, int RS, bool DEFER = false>
__device__ __forceinline__ void stream_step(PencilWindow<T, (RS & 4) ? 6 : 5>& S, int k, const T* Us, const T* old,
                                            T* base, long sAx, const int* comp, T dtdx, const Gas<T>& gs,
                                            const DevMesh& m, const SweepParams& prm, int leaf, int axis,
                                            bool face_row, int pa, int pb, T* upd = nullptr) {
  constexpr int G = kGhosts, N = NB + 2 * G;
  constexpr long SLAB = (long)N * N * N;
  constexpr int NQ = (RS & 4) ? 6 : 5;
  if constexpr (NQ == 6) to_primitive_de(Us, gs, S.w[4]);
  else to_primitive(Us, gs, S.w[4]);
  if (k >= 3 && k <= N - 2) {
#pragma unroll
    for (int c = 0; c < NQ; ++c) S.dm[1][c] = limited_slope(S.w[2][c], S.w[3][c], S.w[4][c]);
  }
  if (k >= 4) {
    S.ft[2] = flatten_tilde(S.w[0][4], S.w[1][4], S.w[3][4], S.w[4][4], S.w[1][1], S.w[3][1]);
    if (RS & 2)
      S.eta[2] = steepening_eta(S.w[0][0], S.w[1][0], S.w[2][0], S.w[3][0], S.w[4][0], S.w[1][4], S.w[3][4], gs.gamma);
    if (k <= N - 2) {
#pragma unroll
      for (int c = 0; c < NQ; ++c)
        S.ai[2][c] = interface_value(S.w[2][c], S.w[3][c], S.dm[0][c], S.dm[1][c]);
    }
  }
  if (k >= 6) {
    // cell j = k-3: W = w[1], aL = ai[0], aR = ai[1], shock detectors ft[0..2]
    const T s = S.w[2][4] - S.w[0][4];
    const T f = (s > T(0)) ? vmax(S.ft[1], S.ft[0]) : ((s < T(0)) ? vmax(S.ft[1], S.ft[2]) : S.ft[1]);
    T aL[NQ], aR[NQ], Wm[NQ], Wp[NQ];
#pragma unroll
    for (int c = 0; c < NQ; ++c) {
      aL[c] = S.ai[0][c];
      aR[c] = S.ai[1][c];
      if ((RS & 2) && c == 0) {   // density of cell k-3: neighbours k-4 (slope dr[0]) and k-2 (slope dm[0])
        const T e = S.eta[1];
        aL[0] = aL[0] * (T(1) - e) + (S.w[0][0] + T(0.5) * S.dr[0]) * e;
        aR[0] = aR[0] * (T(1) - e) + (S.w[2][0] - T(0.5) * S.dm[0][0]) * e;
      }
      flatten_monotone(S.w[1][c], f, aL[c], aR[c]);
    }
    trace<T, NQ>(S.w[1], aL, aR, dtdx, gs, Wm, Wp);
    if (k >= 7) {
      // interface j = k-4 (+1/2): left state wp (cell k-4), right state Wm (cell k-3)
      T F[NQ];
      T uf = T(0);
      if constexpr (NQ == 6) interface_flux6<RS>(S.wp, Wm, gs, F, &uf);
      else interface_flux<RS>(S.wp, Wm, gs, F);
      const int j = k - 4;
      if (face_row && (j == G - 1 || j == G + NB - 1)) {
        const int face = 2 * axis + (j == G - 1 ? 0 : 1);
        const int slot = m.face_slot[leaf * 6 + face];
        if (slot >= 0) {
          double* r = prm.reg + (long)slot * NQ * NB * NB + (pa - G) * NB + (pb - G);
#pragma unroll
          for (int c = 0; c < NQ; ++c) r[(long)comp[c] * NB * NB] = double(F[c]);
        }
      }
      if (k >= 8) {
        // cell j = k-4 (window slot w[0]) between interfaces j-1/2 (fl) and j+1/2 (F)
        T v[NQ];
#pragma unroll
        for (int c = 0; c < NQ; ++c) v[c] = old[c] - dtdx * sub_rn(F[c], S.fl[c]);
        if constexpr (NQ == 6) {
          v[5] = v[5] - (dtdx * S.w[0][4]) * sub_rn(uf, S.ufl);
          v[5] = dual_sync(v);
        }
#pragma unroll
        for (int c = 0; c < NQ; ++c) {
          if (DEFER) upd[c] = v[c];
          else base[comp[c] * SLAB + (long)j * sAx] = v[c];
        }
      }
#pragma unroll
      for (int c = 0; c < NQ; ++c) S.fl[c] = F[c];
      if constexpr (NQ == 6) S.ufl = uf;
    }
#pragma unroll
    for (int c = 0; c < NQ; ++c) S.wp[c] = Wp[c];
  }
  // slide the windows
  if (RS & 2) {
    S.eta[0] = S.eta[1]; S.eta[1] = S.eta[2];
    S.dr[0] = S.dr[1]; S.dr[1] = S.dm[0][0];
  }
#pragma unroll
  for (int c = 0; c < NQ; ++c) {
    S.w[0][c] = S.w[1][c]; S.w[1][c] = S.w[2][c]; S.w[2][c] = S.w[3][c]; S.w[3][c] = S.w[4][c];
    S.dm[0][c] = S.dm[1][c];
    S.ai[0][c] = S.ai[1][c]; S.ai[1][c] = S.ai[2][c];
  }
  S.ft[0] = S.ft[1]; S.ft[1] = S.ft[2];
}

// Float32 form of stream_step: the same quantities at the same cells, the
// fields of each in lane-pair groups (stream_x2.cuh).
template <typename T, int NB, int RS, bool DEFER = false>
__device__ __forceinline__ void stream_step(px::Window<(RS & 4) ? 6 : 5>& S, int k, const float* Us,
                                            const float* old, float* base, long sAx, const int* comp, float dtdx,
                                            const Gas<float>& gs, const DevMesh& m, const SweepParams& prm,
                                            int leaf, int axis, bool face_row, int pa, int pb,
                                            float* upd = nullptr) {
  constexpr int G = kGhosts, N = NB + 2 * G;
  constexpr long SLAB = (long)N * N * N;
  constexpr int NQ = (RS & 4) ? 6 : 5;
  using C = px::Cell<NQ>;
  using CT = typename C::CT;
  S.w[4] = px::primitives<NQ>(Us, gs);
  if (k >= 3 && k <= N - 2)
    S.dm[1] = px::each([](auto am, auto a0, auto ap) { return px::slope(am, a0, ap); }, S.w[2], S.w[3], S.w[4]);
  if (k >= 4) {
    S.ft[2] = flatten_tilde(S.w[0].a.y, S.w[1].a.y, S.w[3].a.y, S.w[4].a.y, S.w[1].a.x, S.w[3].a.x);
    if (RS & 2)
      S.eta[2] = px::steepening(px::lo(S.w[0].c), px::lo(S.w[1].c), px::lo(S.w[2].c), px::lo(S.w[3].c),
                                px::lo(S.w[4].c), S.w[1].a.y, S.w[3].a.y, gs.gamma);
    if (k <= N - 2)
      S.ai[2] = px::each([](auto a0, auto a1, auto d0, auto d1) { return px::interface_val(a0, a1, d0, d1); },
                         S.w[2], S.w[3], S.dm[0], S.dm[1]);
  }
  if (k >= 6) {
    // cell j = k-3: W = w[1], aL = ai[0], aR = ai[1], shock detectors ft[0..2]
    const float s = S.w[2].a.y - S.w[0].a.y;
    const float f = (s > 0.0f) ? vmax(S.ft[1], S.ft[0]) : ((s < 0.0f) ? vmax(S.ft[1], S.ft[2]) : S.ft[1]);
    C aL = S.ai[0], aR = S.ai[1];
    if (RS & 2) {   // density of cell k-3: neighbours k-4 (slope dr[0]) and k-2 (slope dm[0])
      const float e = S.eta[1], ome = px::sub(1.0f, e);
      const float l0 = px::fma(px::lo(aL.c), ome, px::mul(px::fma(0.5f, S.dr[0], px::lo(S.w[0].c)), e));
      const float r0 = px::fma(px::lo(aR.c), ome, px::mul(px::fma(-0.5f, px::lo(S.dm[0].c), px::lo(S.w[2].c)), e));
      if constexpr (NQ == 6) { aL.c.x = l0; aR.c.x = r0; } else { aL.c = l0; aR.c = r0; }
    }
    const float2 f2 = px::splat<float2>(f), omf2 = px::splat<float2>(px::sub(1.0f, f));
    px::flatten_mono(S.w[1].a, f2, omf2, aL.a, aR.a);
    px::flatten_mono(S.w[1].b, f2, omf2, aL.b, aR.b);
    px::flatten_mono(S.w[1].c, px::pick<CT>(f2), px::pick<CT>(omf2), aL.c, aR.c);
    C Wm, Wp;
    px::trace_cell<NQ>(S.w[1], aL, aR, px::splat<float2>(dtdx), gs, Wm, Wp);
    if (k >= 7) {
      // interface j = k-4 (+1/2): left state wp (cell k-4), right state Wm (cell k-3)
      C Fc;
      float uf = 0.0f;
      px::flux<NQ, RS>(S.wp, Wm, gs, Fc, &uf);
      const int j = k - 4;
      if (face_row && (j == G - 1 || j == G + NB - 1)) {
        const int face = 2 * axis + (j == G - 1 ? 0 : 1);
        const int slot = m.face_slot[leaf * 6 + face];
        if (slot >= 0) {
          double* r = prm.reg + (long)slot * NQ * NB * NB + (pa - G) * NB + (pb - G);
#pragma unroll
          for (int c = 0; c < NQ; ++c) r[(long)comp[c] * NB * NB] = double(Fc.get(c));
        }
      }
      if (k >= 8) {
        // cell j = k-4 (window slot w[0]) between interfaces j-1/2 (fl) and j+1/2 (F)
        C o;
#pragma unroll
        for (int c = 0; c < NQ; ++c) o.set(c, old[c]);
        const float2 nd = px::splat<float2>(-dtdx);
        C v;
        v.a = px::fma(nd, px::sub(Fc.a, S.fl.a), o.a);
        v.b = px::fma(nd, px::sub(Fc.b, S.fl.b), o.b);
        v.c = px::fma(px::pick<CT>(nd), px::sub(Fc.c, S.fl.c), o.c);
        if constexpr (NQ == 6) {
          v.c.y = px::fma(-px::mul(dtdx, S.w[0].a.y), px::sub(uf, S.ufl), v.c.y);
          float vv[6];
#pragma unroll
          for (int c = 0; c < 6; ++c) vv[c] = v.get(c);
          v.c.y = px::dual_sync6(vv);
        }
#pragma unroll
        for (int c = 0; c < NQ; ++c) {
          if (DEFER) upd[c] = v.get(c);
          else base[comp[c] * SLAB + (long)j * sAx] = v.get(c);
        }
      }
      S.fl = Fc;
      if constexpr (NQ == 6) S.ufl = uf;
    }
    S.wp = Wp;
  }
  // slide the windows
  if (RS & 2) {
    S.eta[0] = S.eta[1]; S.eta[1] = S.eta[2];
    S.dr[0] = S.dr[1]; S.dr[1] = px::lo(S.dm[0].c);
  }
  S.w[0] = S.w[1]; S.w[1] = S.w[2]; S.w[2] = S.w[3]; S.w[3] = S.w[4];
  S.dm[0] = S.dm[1];
  S.ai[0] = S.ai[1]; S.ai[1] = S.ai[2];
  S.ft[0] = S.ft[1]; S.ft[1] = S.ft[2];
}

// The window type of the streaming sweep: float32 keeps its fields in lane
// pairs.
template <typename T, int NQ> struct WindowOf { using type = PencilWindow<T, NQ>; };
template <int NQ> struct WindowOf<float, NQ> { using type = px::Window<NQ>; };

__device__ __forceinline__ float lane4(const float4& v, int i) {
  return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}


// VEC = 3 (float32, used on the x sweep, whose pencils run along the
// contiguous axis): cells are read and written four at a time as 16-byte
// vectors (a group is read one group ahead; the group updated during group
// g is g-1, written back at its end) instead of 4-byte accesses 160 bytes
// apart across the warp, the groups staged in shared memory by asynchronous
// copies and run two cells per copy of the step; other axes, and VEC = 0,
// take the one-cell walk.
template <typename T, int NB, int CT, int MINB, int VEC, int RS>
__global__ void __launch_bounds__(CT, MINB)
sweep_stream_kernel(DevMesh m, SweepParams prm) {
  constexpr int G = kGhosts, N = NB + 2 * G;
  constexpr long SLAB = (long)N * N * N;
  constexpr int NQ = (RS & 4) ? 6 : 5;   // dual energy: a sixth field rho e
  const Gas<T> gs = Gas<T>::make(m.gamma);
  T* U = static_cast<T*>(prm.U);
  const int axis = prm.axis;
  const int cA = prm.a1 - prm.a0, cB = prm.b1 - prm.b0;
  const long sTA = axis == 2 ? N : (long)N * N;
  const long sTB = axis == 0 ? N : 1;
  int comp[6];
  comp[0] = 0; comp[1] = 1 + axis; comp[4] = 4; comp[5] = 5;
  comp[2] = axis == 0 ? 2 : 1;
  comp[3] = axis == 2 ? 2 : 3;

  const int t = threadIdx.x;
  __shared__ int s_item;
  __shared__ T s_dtdx[16];
  if (t <= m.max_level) s_dtdx[t] = T(*prm.dt / ldexp(m.dx0, -t));
  __syncthreads();

  int item = blockIdx.x;
  if (prm.work) {
    if (t == 0) s_item = (int)atomicAdd(prm.work, 1u);
    __syncthreads();
    item = s_item;
  }
  while (item < prm.n_items) {
    const int lrel = (int)prm.div_tiles.div((unsigned)item);
    const int leaf = prm.leaf0 + lrel;
    const int tile = item - lrel * prm.tiles_per_leaf;
    const int4 lf = m.leaf[leaf];
    const T dtdx = s_dtdx[lf.x];
    const int q = tile * CT + t;
    if (q < cA * cB) {
      const int qa = (int)prm.div_cb.div((unsigned)q);
      const int pa = prm.a0 + qa, pb = prm.b0 + q - qa * cB;
      T* base = U + (long)leaf * NQ * SLAB + pa * sTA + pb * sTB;
      const bool face_row = prm.reg && pa >= G && pa < G + NB && pb >= G && pb < G + NB;
      typename WindowOf<T, NQ>::type S;
      T old[NQ];
      if (VEC == 3 && axis == 0) {
        // the groups of four cells are copied HBM -> shared memory by cp.async, one group
        // ahead, into three per-thread slots (current group, the group being updated, the
        // group in flight); the four cells of a group run through the step two at a time
        // (two copies of the step: half the sliding window's register moves, while four
        // copies would miss in the instruction cache), each updated cell written to a
        // fourth slot that cp.async never targets and stored from there as one vector
        // per field
        extern __shared__ __align__(16) unsigned char stream_raw[];
        float4* my = reinterpret_cast<float4*>(stream_raw) + t;   // slot s, field c at my[(s * NQ + c) * CT]
        const float4* b4 = reinterpret_cast<const float4*>(base);
        constexpr int NG = N / 4;
        auto issue = [&](int grp, int slot) {
#pragma unroll
          for (int c = 0; c < NQ; ++c) {
            const unsigned dst = (unsigned)__cvta_generic_to_shared(&my[(slot * NQ + c) * CT]);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(b4 + comp[c] * (SLAB / 4) + grp)
                         : "memory");
          }
        };
        issue(0, 0);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
#pragma unroll 1
        for (int g = 0; g < NG; ++g) {
          if (g + 1 < NG) issue(g + 1, (g + 1) % 3);
          asm volatile("cp.async.commit_group;\n" ::: "memory");
          asm volatile("cp.async.wait_group 1;\n" ::: "memory");   // group g has landed
          const float* cur = reinterpret_cast<const float*>(my + (g % 3) * NQ * CT);
          const float* prv = reinterpret_cast<const float*>(my + ((g + 2) % 3) * NQ * CT);
          float* out = reinterpret_cast<float*>(my + 3 * NQ * CT);
#pragma unroll 2
          for (int i = 0; i < 4; ++i) {
            T Us[NQ], up[NQ];
#pragma unroll
            for (int c = 0; c < NQ; ++c) {
              Us[c] = cur[c * CT * 4 + i];
              old[c] = prv[c * CT * 4 + i];
            }
            stream_step<T, NB, RS, true>(S, 4 * g + i, Us, old, base, 1, comp, dtdx, gs, m, prm, leaf, axis,
                                         face_row, pa, pb, up);
            if (g >= 2) {   // cells k >= 8: up holds cell 4(g-1)+i
#pragma unroll
              for (int c = 0; c < NQ; ++c) out[c * CT * 4 + i] = up[c];
            }
          }
          if (g >= 2 && g - 1 <= NG - 2) {   // group g-1 holds interior cells 4(g-1) .. 4(g-1)+3
            float4* w4 = reinterpret_cast<float4*>(base);
            const float4* done = my + 3 * NQ * CT;
#pragma unroll
            for (int c = 0; c < NQ; ++c) w4[comp[c] * (SLAB / 4) + g - 1] = done[c * CT];
          }
        }
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
      } else {
        // the one-cell walk, compiled once per axis so that the slab offsets of the fields
        // and the stride along the pencil are constants of the address arithmetic
        auto walk = [&](auto axis_tag) {
          constexpr int AX = decltype(axis_tag)::value;
          constexpr long sA = AX == 0 ? 1 : (AX == 1 ? N : (long)N * N);
          constexpr int cmp[6] = {0, 1 + AX, AX == 0 ? 2 : 1, AX == 2 ? 2 : 3, 4, 5};
          T nx[NQ];   // cell k+1, loaded one step ahead
#pragma unroll
          for (int c = 0; c < NQ; ++c) nx[c] = base[cmp[c] * SLAB];
#pragma unroll 2
          for (int k = 0; k < N; ++k) {
            T Us[NQ];
#pragma unroll
            for (int c = 0; c < NQ; ++c) Us[c] = nx[c];
            if (k + 1 < N) {
#pragma unroll
              for (int c = 0; c < NQ; ++c) nx[c] = base[cmp[c] * SLAB + (k + 1) * sA];
            }
            if (k >= 8) {
#pragma unroll
              for (int c = 0; c < NQ; ++c) old[c] = base[cmp[c] * SLAB + (k - 4) * sA];
            }
            stream_step<T, NB, RS>(S, k, Us, old, base, sA, cmp, dtdx, gs, m, prm, leaf, AX, face_row, pa, pb);
          }
        };
        if (axis == 0) walk(std::integral_constant<int, 0>());
        else if (axis == 1) walk(std::integral_constant<int, 1>());
        else walk(std::integral_constant<int, 2>());
      }
    }
    if (prm.work) {
      __syncthreads();
      if (t == 0) s_item = (int)atomicAdd(prm.work, 1u);
      __syncthreads();
      item = s_item;
    } else {
      item += gridDim.x;
    }
  }
}

// =====================================================================
// Ghost refresh: one thread per ghost cell of a leaf, all NF fields (five,
// or six with the dual-energy formalism's rho e).
// =====================================================================
template <int NB>
__device__ __forceinline__ void ghost_coord(int q, int& x, int& y, int& z) {
  constexpr int G = kGhosts, N = NB + 2 * G, plane = N * N, ring = N * N - NB * NB;
  if (q < G * plane) {
    z = q / plane; const int r = q % plane; y = r / N; x = r % N;
  } else if (q < 2 * G * plane) {
    q -= G * plane; z = G + NB + q / plane; const int r = q % plane; y = r / N; x = r % N;
  } else {
    q -= 2 * G * plane; z = G + q / ring; int r = q % ring;
    if (r < G * N) {
      y = r / N; x = r % N;
    } else if (r < 2 * G * N) {
      r -= G * N; y = G + NB + r / N; x = r % N;
    } else {
      r -= 2 * G * N; y = G + r / (2 * G); const int tt = r % (2 * G); x = tt < G ? tt : NB + tt;
    }
  }
}

// Mean of the 8 cells (fine padded coords f0 + {0,1}^3) of leaf `leaf`,
// summed in (dz, dy, dx) order, times 0.125.
template <typename T, int NB, int NF = 5>
__device__ __forceinline__ void restrict8(const T* U, int leaf, int fx, int fy, int fz, T out[NF]) {
  constexpr int N = NB + 2 * kGhosts;
  constexpr long SLAB = (long)N * N * N;
  const T* b = U + (long)leaf * NF * SLAB + ((long)fz * N + fy) * N + fx;
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const T* c = b + f * SLAB;
    T v = c[0];
    v = v + c[1];
    v = v + c[N];
    v = v + c[N + 1];
    v = v + c[N * N];
    v = v + c[N * N + 1];
    v = v + c[N * N + N];
    v = v + c[N * N + N + 1];
    out[f] = v * T(0.125);
  }
}

template <typename T, int NB, int NF = 5>
__device__ __forceinline__ void load5(const T* U, int leaf, int x, int y, int z, T out[NF]) {
  constexpr int N = NB + 2 * kGhosts;
  constexpr long SLAB = (long)N * N * N;
  const T* b = U + (long)leaf * NF * SLAB + ((long)z * N + y) * N + x;
#pragma unroll
  for (int f = 0; f < NF; ++f) out[f] = b[f * SLAB];
}

// Value of the level-(L-1) cell r (local to the coarse leaf C, r[a] may be
// -1 or NB on exactly one axis a) used as a prolongation slope neighbour:
// C's own cell, a same-level copy, a restriction from level-L leaves, an
// injection from the level-(L-2) leaf, or C's cell itself behind an outflow
// boundary.
template <typename T, int NB, int NF = 5>
__device__ void slope_neighbour(const DevMesh& m, const T* U, int C, const int rc[3], int a, int side,
                                const T Uc[NF], T out[NF]) {
  constexpr int G = kGhosts, H = NB / 2;
  const int fe = face_dir(a, side);
  const int e = C * 27 + fe;
  const int8_t k = m.kind[e];
  if (k == kBoundary) {
#pragma unroll
    for (int f = 0; f < NF; ++f) out[f] = Uc[f];
    return;
  }
  int r2[3] = {rc[0], rc[1], rc[2]};
  r2[a] = side < 0 ? NB - 1 : 0;   // position inside the neighbour node
  if (k == kSame) {
    load5<T, NB, NF>(U, m.idx[e], r2[0] + G, r2[1] + G, r2[2] + G, out);
  } else if (k == kFine) {
    const int o0 = r2[0] / H, o1 = r2[1] / H, o2 = r2[2] / H;
    const int child = m.fine8[e * 8 + o2 * 4 + o1 * 2 + o0];
    restrict8<T, NB, NF>(U, child, 2 * r2[0] - o0 * NB + G, 2 * r2[1] - o1 * NB + G, 2 * r2[2] - o2 * NB + G, out);
  } else {  // coarser: inject the level-(L-2) cell
    const int4 cl = m.leaf[C];
    const int K = m.idx[e];
    const int4 kl = m.leaf[K];
    const int Lc = cl.x;
    int g[3] = {cl.y * NB + rc[0], cl.z * NB + rc[1], cl.w * NB + rc[2]};
    g[a] += side;
    const int ncell = (m.root[a] << Lc) * NB;
    g[a] = wrap_mod(g[a], ncell);
    const int lx = (g[0] >> 1) - kl.y * NB, ly = (g[1] >> 1) - kl.z * NB, lz = (g[2] >> 1) - kl.w * NB;
    load5<T, NB, NF>(U, K, lx + G, ly + G, lz + G, out);
  }
}

// Value of one ghost cell (padded coords c, already inside the block
// array) of leaf `leaf`: same-level copy, restriction or prolongation.
template <typename T, int NB, int NF = 5>
__device__ void ghost_value(const DevMesh& m, const T* U, int leaf, int c[3], T v[NF]) {
  constexpr int G = kGhosts, H = NB / 2;
  int d[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    d[a] = c[a] < G ? -1 : (c[a] >= G + NB ? 1 : 0);
    if (d[a] != 0 && m.kind[leaf * 27 + face_dir(a, d[a])] == kBoundary) {
      c[a] = d[a] < 0 ? G : G + NB - 1;   // outflow: nearest interior cell
      d[a] = 0;
    }
  }
  const int e = leaf * 27 + (d[2] + 1) * 9 + (d[1] + 1) * 3 + (d[0] + 1);
  const int8_t k = m.kind[e];
  if (k == kSame) {
    load5<T, NB, NF>(U, m.idx[e], c[0] - d[0] * NB, c[1] - d[1] * NB, c[2] - d[2] * NB, v);
  } else if (k == kFine) {
    int r[3], o[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      r[a] = c[a] - G - d[a] * NB;
      o[a] = r[a] / H;
    }
    const int child = m.fine8[e * 8 + o[2] * 4 + o[1] * 2 + o[0]];
    restrict8<T, NB, NF>(U, child, 2 * r[0] - o[0] * NB + G, 2 * r[1] - o[1] * NB + G, 2 * r[2] - o[2] * NB + G, v);
  } else {  // coarse: conservative minmod-limited linear prolongation
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
    T Uc[NF];
    load5<T, NB, NF>(U, C, rc[0] + G, rc[1] + G, rc[2] + G, Uc);
    T D[3][NF];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      T Um[NF], Up[NF];
      int rm[3] = {rc[0], rc[1], rc[2]}, rp[3] = {rc[0], rc[1], rc[2]};
      rm[a] -= 1;
      rp[a] += 1;
      if (rm[a] >= 0) load5<T, NB, NF>(U, C, rm[0] + G, rm[1] + G, rm[2] + G, Um);
      else slope_neighbour<T, NB, NF>(m, U, C, rc, a, -1, Uc, Um);
      if (rp[a] < NB) load5<T, NB, NF>(U, C, rp[0] + G, rp[1] + G, rp[2] + G, Up);
      else slope_neighbour<T, NB, NF>(m, U, C, rc, a, 1, Uc, Up);
#pragma unroll
      for (int f = 0; f < NF; ++f) D[a][f] = minmod(Uc[f] - Um[f], Up[f] - Uc[f]);
    }
#pragma unroll
    for (int f = 0; f < NF; ++f)
      v[f] = Uc[f] + T(0.25) * ((sgn[0] * D[0][f] + sgn[1] * D[1][f]) + sgn[2] * D[2][f]);
  }
}

// 16-byte vector of four consecutive cells.
template <typename T> struct Vec4;
template <> struct Vec4<float> {
  float4 a;
  __device__ __forceinline__ void load(const float* p) { a = *reinterpret_cast<const float4*>(p); }
  __device__ __forceinline__ void store(float* p) const { *reinterpret_cast<float4*>(p) = a; }
};
template <> struct Vec4<double> {
  double2 a, b;
  __device__ __forceinline__ void load(const double* p) {
    a = reinterpret_cast<const double2*>(p)[0];
    b = reinterpret_cast<const double2*>(p)[1];
  }
  __device__ __forceinline__ void store(double* p) const {
    reinterpret_cast<double2*>(p)[0] = a;
    reinterpret_cast<double2*>(p)[1] = b;
  }
};
__device__ __forceinline__ void store_lanes(const Vec4<float>& v, float* o) {
  o[0] = v.a.x; o[1] = v.a.y; o[2] = v.a.z; o[3] = v.a.w;
}
__device__ __forceinline__ void store_lanes(const Vec4<double>& v, double* o) {
  o[0] = v.a.x; o[1] = v.a.y; o[2] = v.b.x; o[3] = v.b.y;
}
__device__ __forceinline__ void load_lanes(Vec4<float>& v, const float* o) {
  v.a = make_float4(o[0], o[1], o[2], o[3]);
}
__device__ __forceinline__ void load_lanes(Vec4<double>& v, const double* o) {
  v.a = make_double2(o[0], o[1]);
  v.b = make_double2(o[2], o[3]);
}

// One 32-byte DRAM sector of consecutive cells (8 floats or 4 doubles),
// moved by a single 256-bit access: a sector written whole by one store is
// not read from DRAM first, which a store of half a sector would cause.
// The address must be 32-byte aligned.
template <typename T> struct Sector;
template <> struct Sector<float> {
  static constexpr int kCells = 8;
  float v[8];
  __device__ __forceinline__ void load(const float* p) {
    asm volatile("ld.global.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
                 : "l"(p));
  }
  __device__ __forceinline__ void store(float* p) const {
    asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(v[0]), "f"(v[1]),
                 "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
                 : "memory");
  }
};
template <> struct Sector<double> {
  static constexpr int kCells = 4;
  double v[4];
  __device__ __forceinline__ void load(const double* p) {
    asm volatile("ld.global.v4.f64 {%0, %1, %2, %3}, [%4];" : "=d"(v[0]), "=d"(v[1]), "=d"(v[2]), "=d"(v[3]) : "l"(p));
  }
  __device__ __forceinline__ void store(double* p) const {
    asm volatile("st.global.v4.f64 [%0], {%1, %2, %3, %4};" ::"l"(p), "d"(v[0]), "d"(v[1]), "d"(v[2]), "d"(v[3])
                 : "memory");
  }
};

// The refresh runs in three phases, one per axis, each a copy across the
// faces of that axis from same-level face neighbours:
//   X: the x margins of interior rows (y and z interior);
//   Y: the y-ghost rows of interior z planes, all N cells of each row;
//   Z: the z-ghost planes, all N x N cells of each.
// A ghost cell's value depends only on its position and level (the level-L
// cell there after the boundary rule), so the margins of a face neighbour's
// rows, filled by an earlier phase, are exactly the edge and corner ghosts
// of this leaf: Y copies whole rows (x margins included) and Z whole planes.
// A face whose neighbour is not a same-level leaf (coarser, finer, outflow
// boundary) has its phase region listed as slow work, computed from leaf
// interiors.
//
// Phase X: the x margins of the interior rows, every access one whole
// 32-byte sector.  A margin fills its sector only in float64; in float32 it is
// half of the sector it shares with the adjacent interior run, and the two
// halves of an exchange are written together: across the face between a
// left leaf L and a right leaf R, the sectors L[row][NB, NB+8) and
// R[row][0, 8) both become (L's last interior run, R's first interior run).
//
// float32: the last sector of row y and the first of row y+1 are one 64-byte
// DRAM unit, so one thread per (leaf A, interior z, row pair y = G + 2k, y + 1)
// owns that unit: it exchanges A's +x face at row y and A's -x face at row
// y+1 (each with a same-level neighbour only), reading each partner's sector
// once.  The +x face of the odd rows and the -x face of the even rows are the
// threads of the neighbours.  float64: one thread per (leaf A, interior row)
// exchanges A's -x face (A's +x face is its +x neighbour's thread).  Faces
// whose neighbour is not a same-level leaf are slow work, done before.
template <typename T, int NB, int NF = 5>
__global__ void __launch_bounds__(256) refresh_x_kernel(DevMesh m, T* U, int leaf0, int nleaf) {
  constexpr int G = kGhosts, N = NB + 2 * G;
  constexpr long SLAB = (long)N * N * N;
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if constexpr (sizeof(T) == 4) {
    constexpr int H = NB / 2;
    if (gid >= (long)nleaf * NB * H) return;
    const int A = leaf0 + (int)(gid / (NB * H));
    const int r = (int)(gid % (NB * H));
    const int y = G + 2 * (r % H), z = G + r / H;
    const int ep = A * 27 + face_dir(0, 1), em = A * 27 + face_dir(0, -1);
    const bool xp = m.kind[ep] == kSame, xm = m.kind[em] == kSame;
    if (!xp && !xm) return;
    const long row = ((long)z * N + y) * N;   // row y; row y + 1 starts at row + N
    T* a = U + (long)A * NF * SLAB + row;
    T* bp = xp ? U + (long)m.idx[ep] * NF * SLAB + row : nullptr;          // right neighbour, row y
    T* bm = xm ? U + (long)m.idx[em] * NF * SLAB + row + N : nullptr;      // left neighbour, row y + 1
#pragma unroll 1
    for (int f = 0; f < NF; ++f) {
      Sector<T> u0, u1, sp, sm;
      u0.load(a + f * SLAB + NB);       // A[y][NB, NB+8): interior run, +x margin
      u1.load(a + f * SLAB + N);        // A[y+1][0, 8): -x margin, interior run
      if (xp) sp.load(bp + f * SLAB);   // R[y][0, 8)
      if (xm) sm.load(bm + f * SLAB + NB);   // L[y+1][NB, NB+8)
      if (xp) {
        Sector<T> o;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          o.v[i] = u0.v[i];
          o.v[4 + i] = sp.v[4 + i];
        }
        o.store(a + f * SLAB + NB);
        o.store(bp + f * SLAB);
      }
      if (xm) {
        Sector<T> o;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          o.v[i] = sm.v[i];
          o.v[4 + i] = u1.v[4 + i];
        }
        o.store(a + f * SLAB + N);
        o.store(bm + f * SLAB + NB);
      }
    }
  } else {
    if (gid >= (long)nleaf * NB * NB) return;
    const int A = leaf0 + (int)(gid / (NB * NB));
    const int r = (int)(gid % (NB * NB));
    const int e = A * 27 + face_dir(0, -1);
    if (m.kind[e] != kSame) return;
    const long row = ((long)(G + r / NB) * N + (G + r % NB)) * N;
    T* a = U + (long)A * NF * SLAB + row;
    T* b = U + (long)m.idx[e] * NF * SLAB + row;
    Sector<T> sa[NF], sb[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      sa[f].load(a + f * SLAB + G);    // A's first interior run
      sb[f].load(b + f * SLAB + NB);   // B's last interior run
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      sb[f].store(a + f * SLAB);          // A's -x margin
      sa[f].store(b + f * SLAB + G + NB); // B's +x margin
    }
  }
}

// Phase Y: one thread per (leaf, side, field, interior z, sector of the G
// rows of that side), copying from the same-level y neighbour C's G interior
// rows next to the face; the G rows of one z plane are contiguous (G N
// cells, whole sectors).
template <typename T, int NB, int NF = 5>
__global__ void __launch_bounds__(256) refresh_y_kernel(DevMesh m, T* U, int leaf0, int nleaf) {
  constexpr int G = kGhosts, N = NB + 2 * G, S = Sector<T>::kCells, RUNS = G * N / S;
  constexpr long SLAB = (long)N * N * N;
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long)nleaf * 2 * NF * NB * RUNS) return;
  long q = gid;
  const int v = (int)(q % RUNS); q /= RUNS;
  const int z = G + (int)(q % NB); q /= NB;
  const int f = (int)(q % NF); q /= NF;
  const int side = (int)(q % 2) ? 1 : -1;
  const int leaf = leaf0 + (int)(q / 2);
  const int e = leaf * 27 + face_dir(1, side);
  if (m.kind[e] != kSame) return;
  const int C = m.idx[e];
  const int yd = side < 0 ? 0 : G + NB, ys = side < 0 ? NB : G;
  Sector<T> t;
  t.load(U + (long)C * NF * SLAB + f * SLAB + ((long)z * N + ys) * N + S * v);
  t.store(U + (long)leaf * NF * SLAB + f * SLAB + ((long)z * N + yd) * N + S * v);
}

// Phase Z: one thread per (leaf, side, field, sector of the G planes of that
// side), copying from the same-level z neighbour's G interior planes next to
// the face (G N N contiguous cells).
template <typename T, int NB, int NF = 5>
__global__ void __launch_bounds__(256) refresh_z_kernel(DevMesh m, T* U, int leaf0, int nleaf) {
  constexpr int G = kGhosts, N = NB + 2 * G, S = Sector<T>::kCells, RUNS = G * N * N / S;
  constexpr long SLAB = (long)N * N * N;
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long)nleaf * 2 * NF * RUNS) return;
  long q = gid;
  const int v = (int)(q % RUNS); q /= RUNS;
  const int f = (int)(q % NF); q /= NF;
  const int side = (int)(q % 2) ? 1 : -1;
  const int leaf = leaf0 + (int)(q / 2);
  const int e = leaf * 27 + face_dir(2, side);
  if (m.kind[e] != kSame) return;
  const int C = m.idx[e];
  const int zd = side < 0 ? 0 : G + NB, zs = side < 0 ? NB : G;
  Sector<T> t;
  t.load(U + (long)C * NF * SLAB + f * SLAB + (long)zs * N * N + S * v);
  t.store(U + (long)leaf * NF * SLAB + f * SLAB + (long)zd * N * N + S * v);
}

// Runs of four cells (x0 .. x0+3, y, z) in the phase region of one face
// (axis, side) of a leaf: the x margin of the interior rows (X), the G ghost
// rows of the interior z planes (Y), the G ghost planes (Z).
template <int NB>
__host__ __device__ constexpr int face_region_runs(int axis) {
  return axis == 0 ? NB * NB
                   : (axis == 1 ? NB * kGhosts * ((NB + 2 * kGhosts) / 4)
                                : kGhosts * (NB + 2 * kGhosts) * ((NB + 2 * kGhosts) / 4));
}

template <int NB>
__device__ __forceinline__ void face_region_run(int axis, int side, int r, int& x0, int& y, int& z) {
  constexpr int G = kGhosts, N = NB + 2 * G, R = N / 4;
  const int lo = side < 0 ? 0 : G + NB;
  if (axis == 0) {
    x0 = lo; y = G + r % NB; z = G + r / NB;
  } else if (axis == 1) {
    x0 = 4 * (r % R); y = lo + (r / R) % G; z = G + r / (R * G);
  } else {
    x0 = 4 * (r % R); y = (r / R) % N; z = lo + r / (R * N);
  }
}

// One run that is not a phase copy: a run clamped along x repeats one value;
// a run inside a coarser neighbour covers two parent cells, each prolonged
// once for its two children; any other run (restriction from finer leaves,
// or a same-level diagonal source seen through a face that is not
// same-level) is evaluated cell by cell.  Sources are leaf interiors only.
template <typename T, int NB, int NF>
__device__ void refresh_slow_run(const DevMesh& m, T* U, int leaf, int x0, int y, int z) {
  constexpr int G = kGhosts, N = NB + 2 * G;
  constexpr long SLAB = (long)N * N * N;
  const long dst = (long)leaf * NF * SLAB + ((long)z * N + y) * N + x0;
  int d[3] = {x0 < G ? -1 : (x0 >= G + NB ? 1 : 0), y < G ? -1 : (y >= G + NB ? 1 : 0),
              z < G ? -1 : (z >= G + NB ? 1 : 0)};
  int c[3] = {x0, y, z};
  bool xclamp = false;
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (d[a] != 0 && m.kind[leaf * 27 + face_dir(a, d[a])] == kBoundary) {
      c[a] = d[a] < 0 ? G : G + NB - 1;
      d[a] = 0;
      if (a == 0) xclamp = true;
    }
  const int e = leaf * 27 + (d[2] + 1) * 9 + (d[1] + 1) * 3 + (d[0] + 1);
  const int8_t k = m.kind[e];
  if (xclamp) {   // every cell of the run reads the same boundary cell
    int cc[3] = {c[0], c[1], c[2]};
    T v[NF];
    ghost_value<T, NB, NF>(m, U, leaf, cc, v);
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int f = 0; f < NF; ++f) U[dst + q + f * SLAB] = v[f];
    return;
  }
  if (k != kCoarse) {
    for (int q = 0; q < 4; ++q) {
      int cc[3] = {x0 + q, y, z};
      T v[NF];
      ghost_value<T, NB, NF>(m, U, leaf, cc, v);
#pragma unroll
      for (int f = 0; f < NF; ++f) U[dst + q + f * SLAB] = v[f];
    }
    return;
  }
  // coarser neighbour: parents of cells (x0, x0+1) and (x0+2, x0+3)
  const int4 lf = m.leaf[leaf];
  const int C = m.idx[e];
  const int4 cl = m.leaf[C];
  const int L = lf.x;
  const int lij[3] = {lf.y, lf.z, lf.w}, cij[3] = {cl.y, cl.z, cl.w};
  int rcyz[3];
  T sgn[3];
#pragma unroll
  for (int a = 1; a < 3; ++a) {
    const int ncell = (m.root[a] << L) * NB;
    const int gl = wrap_mod(lij[a] * NB + (c[a] - G), ncell);
    rcyz[a] = (gl >> 1) - cij[a] * NB;
    sgn[a] = (gl & 1) ? T(1) : T(-1);
  }
  const int ncx = (m.root[0] << L) * NB;
  for (int h = 0; h < 2; ++h) {
    const int gl = wrap_mod(lij[0] * NB + (x0 + 2 * h - G), ncx);   // even: the lower child
    int rc[3] = {(gl >> 1) - cij[0] * NB, rcyz[1], rcyz[2]};
    T Uc[NF], D[3][NF];
    load5<T, NB, NF>(U, C, rc[0] + G, rc[1] + G, rc[2] + G, Uc);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      T Um[NF], Up[NF];
      int rm[3] = {rc[0], rc[1], rc[2]}, rp[3] = {rc[0], rc[1], rc[2]};
      rm[a] -= 1;
      rp[a] += 1;
      if (rm[a] >= 0) load5<T, NB, NF>(U, C, rm[0] + G, rm[1] + G, rm[2] + G, Um);
      else slope_neighbour<T, NB, NF>(m, U, C, rc, a, -1, Uc, Um);
      if (rp[a] < NB) load5<T, NB, NF>(U, C, rp[0] + G, rp[1] + G, rp[2] + G, Up);
      else slope_neighbour<T, NB, NF>(m, U, C, rc, a, 1, Uc, Up);
#pragma unroll
      for (int f = 0; f < NF; ++f) D[a][f] = minmod(Uc[f] - Um[f], Up[f] - Uc[f]);
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const T sx = q ? T(1) : T(-1);
#pragma unroll
      for (int f = 0; f < NF; ++f)
        U[dst + 2 * h + q + f * SLAB] = Uc[f] + T(0.25) * ((sx * D[0][f] + sgn[1] * D[1][f]) + sgn[2] * D[2][f]);
    }
  }
}

// Quads of runs: runs (x0, y + jy, z + jz), jy, jz in {0, 1}, y and z even,
// so that in each axis the two rows are the two children of one parent row.
// The quads tile the phase region of a face (its extents in y and z are even).
template <int NB>
__host__ __device__ constexpr int face_region_quads(int axis) {
  return face_region_runs<NB>(axis) / 4;
}

template <int NB>
__device__ __forceinline__ void face_region_quad(int axis, int side, int r, int& x0, int& y, int& z) {
  constexpr int G = kGhosts, N = NB + 2 * G, R = N / 4;
  const int lo = side < 0 ? 0 : G + NB;
  if (axis == 0) {
    x0 = lo; y = G + 2 * (r % (NB / 2)); z = G + 2 * (r / (NB / 2));
  } else if (axis == 1) {
    x0 = 4 * (r % R); y = lo + 2 * ((r / R) % (G / 2)); z = G + 2 * (r / (R * (G / 2)));
  } else {
    x0 = 4 * (r % R); y = 2 * ((r / R) % (N / 2)); z = lo + 2 * (r / (R * (N / 2)));
  }
}

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

// One quad of a slow face: all 16 cells lie in one neighbour direction.
// Coarser neighbour: each of the two parents along x is prolonged once for
// its eight children (the per-run path would take its slopes four times);
// finer neighbour: each coarse ghost cell restricts its eight children with
// vector loads of the children's rows.  Outflow clamps and same-level
// diagonal sources take the per-run path.  The arithmetic of every value is
// that of ghost_value (same operations, same order).
template <typename T, int NB, int NF>
__device__ void refresh_slow_quad(const DevMesh& m, T* U, int leaf, int x0, int y, int z) {
  constexpr int G = kGhosts, N = NB + 2 * G, H = NB / 2;
  constexpr long SLAB = (long)N * N * N;
  const int c[3] = {x0, y, z};
  int d[3];
  bool clamp = false;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    d[a] = c[a] < G ? -1 : (c[a] >= G + NB ? 1 : 0);
    if (d[a] != 0 && m.kind[leaf * 27 + face_dir(a, d[a])] == kBoundary) clamp = true;
  }
  const int e = leaf * 27 + (d[2] + 1) * 9 + (d[1] + 1) * 3 + (d[0] + 1);
  const int8_t k = m.kind[e];
  if (clamp || k == kSame) {
    for (int j = 0; j < 4; ++j) refresh_slow_run<T, NB, NF>(m, U, leaf, x0, y + (j & 1), z + (j >> 1));
    return;
  }
  T* const dst = U + (long)leaf * NF * SLAB;
  if (k == kFine) {
    for (int j = 0; j < 4; ++j) {
      const int cy = y + (j & 1), cz = z + (j >> 1);
      const int r[3] = {x0 - G - d[0] * NB, cy - G - d[1] * NB, cz - G - d[2] * NB};
      const int o[3] = {r[0] / H, r[1] / H, r[2] / H};
      const int child = m.fine8[e * 8 + o[2] * 4 + o[1] * 2 + o[0]];
      const int f0 = 2 * r[0] - o[0] * NB + G, f1 = 2 * r[1] - o[1] * NB + G, f2 = 2 * r[2] - o[2] * NB + G;
      const T* src = U + (long)child * NF * SLAB + ((long)f2 * N + f1) * N + f0;
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        // the children's rows (dz, dy) = (0,0), (0,1), (1,0), (1,1), eight cells each
        T v[4][8];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const T* row = src + f * SLAB + (q >> 1) * (long)N * N + (q & 1) * N;
          Vec4<T> lo4, hi4;
          lo4.load(row);
          hi4.load(row + 4);
          store_lanes(lo4, v[q]);
          store_lanes(hi4, v[q] + 4);
        }
        T out[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          T a = v[0][2 * i];
          a = a + v[0][2 * i + 1];
          a = a + v[1][2 * i];
          a = a + v[1][2 * i + 1];
          a = a + v[2][2 * i];
          a = a + v[2][2 * i + 1];
          a = a + v[3][2 * i];
          a = a + v[3][2 * i + 1];
          out[i] = a * T(0.125);
        }
        Vec4<T> w;
        load_lanes(w, out);
        w.store(dst + f * SLAB + ((long)cz * N + cy) * N + x0);
      }
    }
    return;
  }
  // coarser neighbour C: parents (x0, x0 + 1) and (x0 + 2, x0 + 3) along x;
  // rows y, y + 1 and z, z + 1 are the lower and upper children in y and z
  const int4 lf = m.leaf[leaf];
  const int C = m.idx[e];
  const int4 cl = m.leaf[C];
  const int L = lf.x;
  const int lij[3] = {lf.y, lf.z, lf.w}, cij[3] = {cl.y, cl.z, cl.w};
  int rc[3];
#pragma unroll
  for (int a = 1; a < 3; ++a)
    rc[a] = (wrap_mod(lij[a] * NB + (c[a] - G), (m.root[a] << L) * NB) >> 1) - cij[a] * NB;
  const int ncx = (m.root[0] << L) * NB;
  using V2 = typename Vec2<T>::type;
  for (int h = 0; h < 2; ++h) {
    rc[0] = (wrap_mod(lij[0] * NB + (x0 + 2 * h - G), ncx) >> 1) - cij[0] * NB;
    T Uc[NF], D[3][NF];
    load5<T, NB, NF>(U, C, rc[0] + G, rc[1] + G, rc[2] + G, Uc);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      T Um[NF], Up[NF];
      int rm[3] = {rc[0], rc[1], rc[2]}, rp[3] = {rc[0], rc[1], rc[2]};
      rm[a] -= 1;
      rp[a] += 1;
      if (rm[a] >= 0) load5<T, NB, NF>(U, C, rm[0] + G, rm[1] + G, rm[2] + G, Um);
      else slope_neighbour<T, NB, NF>(m, U, C, rc, a, -1, Uc, Um);
      if (rp[a] < NB) load5<T, NB, NF>(U, C, rp[0] + G, rp[1] + G, rp[2] + G, Up);
      else slope_neighbour<T, NB, NF>(m, U, C, rc, a, 1, Uc, Up);
#pragma unroll
      for (int f = 0; f < NF; ++f) D[a][f] = minmod(Uc[f] - Um[f], Up[f] - Uc[f]);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const T sy = (j & 1) ? T(1) : T(-1), sz = (j >> 1) ? T(1) : T(-1);
      T* row = dst + ((long)(z + (j >> 1)) * N + (y + (j & 1))) * N + x0 + 2 * h;
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        V2 w;
        w.x = Uc[f] + T(0.25) * ((T(-1) * D[0][f] + sy * D[1][f]) + sz * D[2][f]);
        w.y = Uc[f] + T(0.25) * ((T(1) * D[0][f] + sy * D[1][f]) + sz * D[2][f]);
        *reinterpret_cast<V2*>(row + f * SLAB) = w;
      }
    }
  }
}

// The slow work, listed per mesh as faces (leaf * 6 + face, faces in the
// order -x, +x, -y, +y, -z, +z) whose neighbour is not a same-level leaf: one
// CTA per listed face, its threads over the quads of that face's phase region.
template <typename T, int NB, int NF = 5>
__global__ void __launch_bounds__(128) refresh_slow_kernel(DevMesh m, T* U, const int* faces, int nfaces) {
  const int i = blockIdx.x;
  if (i >= nfaces) return;
  const int leaf = faces[i] / 6, face = faces[i] % 6;
  const int axis = face >> 1, side = (face & 1) ? 1 : -1;
  const int nq = face_region_quads<NB>(axis);
  for (int r = threadIdx.x; r < nq; r += blockDim.x) {
    int x0, y, z;
    face_region_quad<NB>(axis, side, r, x0, y, z);
    refresh_slow_quad<T, NB, NF>(m, U, leaf, x0, y, z);
  }
}

// =====================================================================
// Remap onto a rebuilt mesh: one thread per interior cell of a new leaf.
// =====================================================================
template <typename T, int NB, int NF = 5>
__global__ void __launch_bounds__(256) remap_kernel(DevMesh neu, DevMesh old, const T* Uold, T* Unew,
                                                    const RemapEntry* map) {
  constexpr int G = kGhosts, N = NB + 2 * G, H = NB / 2;
  constexpr long SLAB = (long)N * N * N;
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long)neu.B * NB * NB * NB) return;
  const int leaf = (int)(gid / (NB * NB * NB));
  const int i = (int)(gid % (NB * NB * NB));
  const int r[3] = {i % NB, (i / NB) % NB, i / (NB * NB)};
  const RemapEntry e = map[leaf];
  T v[NF];
  if (e.kind == 0) {
    load5<T, NB, NF>(Uold, e.src[0], r[0] + G, r[1] + G, r[2] + G, v);
  } else if (e.kind == 2) {
    const int o[3] = {r[0] / H, r[1] / H, r[2] / H};
    restrict8<T, NB, NF>(Uold, e.src[o[2] * 4 + o[1] * 2 + o[0]], 2 * r[0] - o[0] * NB + G, 2 * r[1] - o[1] * NB + G,
                     2 * r[2] - o[2] * NB + G, v);
  } else {
    const int4 nl = neu.leaf[leaf];
    const int4 al = old.leaf[e.src[0]];
    const int k = e.k;
    const int nij[3] = {nl.y, nl.z, nl.w}, aij[3] = {al.y, al.z, al.w};
    int c[3];
    T xi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int gf = nij[a] * NB + r[a];
      c[a] = (gf >> k) - aij[a] * NB + G;
      xi[a] = T((double((gf & ((1 << k) - 1))) + 0.5) / double(1 << k) - 0.5);
    }
    T Uc[NF], D[3][NF];
    load5<T, NB, NF>(Uold, e.src[0], c[0], c[1], c[2], Uc);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      int cm[3] = {c[0], c[1], c[2]}, cp[3] = {c[0], c[1], c[2]};
      cm[a] -= 1;
      cp[a] += 1;
      T Um[NF], Up[NF];
      load5<T, NB, NF>(Uold, e.src[0], cm[0], cm[1], cm[2], Um);
      load5<T, NB, NF>(Uold, e.src[0], cp[0], cp[1], cp[2], Up);
#pragma unroll
      for (int f = 0; f < NF; ++f) D[a][f] = minmod(Uc[f] - Um[f], Up[f] - Uc[f]);
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) v[f] = Uc[f] + ((xi[0] * D[0][f] + xi[1] * D[1][f]) + xi[2] * D[2][f]);
  }
  const long dst = (long)leaf * NF * SLAB + ((long)(r[2] + G) * N + (r[1] + G)) * N + (r[0] + G);
#pragma unroll
  for (int f = 0; f < NF; ++f) Unew[dst + f * SLAB] = v[f];
}

// =====================================================================
// CFL dt candidates and conserved sums, one CTA per leaf at a time (grid-
// stride over the leaves; a leaf's partials do not depend on the grid),
// then a single-CTA fixed-order finish.  Deterministic.
// =====================================================================
constexpr int kReduceThreads = 256;

__device__ __forceinline__ void block_reduce6(double v[6], double* sh) {
  // v[0] min, v[1..5] sums; fixed tree: xor shuffles, then warp 0 over warps.
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v[0] = fmin(v[0], __shfl_xor_sync(0xffffffffu, v[0], o));
#pragma unroll
    for (int k = 1; k < 6; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (l == 0)
#pragma unroll
    for (int k = 0; k < 6; ++k) sh[w * 6 + k] = v[k];
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int k = 0; k < 6; ++k) v[k] = (l < nw) ? sh[l * 6 + k] : (k == 0 ? INFINITY : 0.0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v[0] = fmin(v[0], __shfl_xor_sync(0xffffffffu, v[0], o));
#pragma unroll
      for (int k = 1; k < 6; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    }
  }
}

// NF = 6 (dual energy): the pressure for the sound speed and the health
// check is selected as in the sweep's primitives, from E - ke or from rho e.
template <typename T, int NB, int NF = 5>
__global__ void __launch_bounds__(kReduceThreads) reduce_partials_kernel(DevMesh m, const T* U, double* partials,
                                                                         int leaf0, int nleaf) {
  constexpr int G = kGhosts, N = NB + 2 * G;
  constexpr long SLAB = (long)N * N * N;
  __shared__ double sh[6 * 32];
  for (int lr = blockIdx.x; lr < nleaf; lr += gridDim.x) {
  const int leaf = leaf0 + lr;
  const int4 lf = m.leaf[leaf];
  const T dx = T(ldexp(m.dx0, -lf.x));
  const T gamma = T(m.gamma), gm1 = T(m.gamma - 1.0);
  const T* b = U + (long)leaf * NF * SLAB;
  double v[6] = {INFINITY, 0, 0, 0, 0, 0};
  int bad = 0;
  for (int i = threadIdx.x; i < NB * NB * NB; i += blockDim.x) {
    const int x = i % NB + G, y = (i / NB) % NB + G, z = i / (NB * NB) + G;
    const long o = ((long)z * N + y) * N + x;
    const T r0 = b[o], m1 = b[SLAB + o], m2 = b[2 * SLAB + o], m3 = b[3 * SLAB + o], E = b[4 * SLAB + o];
    const T rho = vmax(r0, T(kRhoFloor));
    const T u = m1 / rho, vv = m2 / rho, w = m3 / rho;
    const T ke = (T(0.5) * rho) * (u * u + (vv * vv + w * w));
    T src = E - ke;
    if constexpr (NF == 6) src = (src > T(kDualEta1) * E) ? src : b[5 * SLAB + o];
    const T praw = gm1 * src;
    bad |= !(r0 > T(0)) || !(praw > T(0)) || !isfinite(praw + (m1 + m2 + m3));
    const T p = vmax(praw, T(kPFloor));
    const T c = vsqrt((gamma * p) / rho);
    const T s = vmax(vabs(u), vmax(vabs(vv), vabs(w))) + c;
    v[0] = fmin(v[0], double(dx / s));
    v[1] += double(r0); v[2] += double(m1); v[3] += double(m2); v[4] += double(m3); v[5] += double(E);
  }
  bad = __syncthreads_or(bad);
  block_reduce6(v, sh);
  if (threadIdx.x == 0) {
    const double dxd = ldexp(m.dx0, -lf.x);
    const double vol = dxd * dxd * dxd;
    partials[leaf * 6 + 0] = v[0];
    for (int k = 1; k < 6; ++k) partials[leaf * 6 + k] = v[k] * vol;
    if (bad && m.err) atomicOr(m.err, 1u);
  }
  __syncthreads();   // sh is rewritten by the next leaf
  }
}

// Float32 state: per-thread sums carried as unevaluated float pairs (Knuth's
// TwoSum keeps each addition's rounding error), the dt candidate minimum in
// float32 (the same value as a float64 minimum of the converted candidates);
// each thread converts once to float64 and the tree runs in float64.
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  const float e = (hi - (s - bp)) + (x - bp);
  hi = s;
  lo += e;
}

template <int NB, int NF = 5>
__global__ void __launch_bounds__(kReduceThreads) reduce_partials_f32_kernel(DevMesh m, const float* U,
                                                                             double* partials, int leaf0, int nleaf) {
  constexpr int G = kGhosts, N = NB + 2 * G;
  constexpr long SLAB = (long)N * N * N;
  __shared__ double sh[6 * 32];
  for (int lr = blockIdx.x; lr < nleaf; lr += gridDim.x) {
  const int leaf = leaf0 + lr;
  const int4 lf = m.leaf[leaf];
  const float dx = float(ldexp(m.dx0, -lf.x));
  const float gamma = float(m.gamma), gm1 = float(m.gamma - 1.0);
  const float* b = U + (long)leaf * NF * SLAB;
  float mn = INFINITY, hi[5] = {0, 0, 0, 0, 0}, lo[5] = {0, 0, 0, 0, 0};
  int bad = 0;
  // four cells along x per 16-byte load (interior rows start at x = G, a
  // multiple of four cells)
  constexpr int Q = NB / 4;
  for (int i = threadIdx.x; i < NB * NB * Q; i += blockDim.x) {
    const int qx = i % Q, row = i / Q;
    const long o = ((long)(row / NB + G) * N + (row % NB + G)) * N + G + 4 * qx;
    float4 v[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) v[f] = *reinterpret_cast<const float4*>(b + f * SLAB + o);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float r0 = lane4(v[0], k), m1 = lane4(v[1], k), m2 = lane4(v[2], k), m3 = lane4(v[3], k),
                  E = lane4(v[4], k);
      const float rho = vmax(r0, float(kRhoFloor));
      const float u = m1 / rho, vv = m2 / rho, w = m3 / rho;
      const float ke = (0.5f * rho) * (u * u + (vv * vv + w * w));
      float src = E - ke;
      if constexpr (NF == 6) src = (src > float(kDualEta1) * E) ? src : lane4(v[NF - 1], k);
      const float praw = gm1 * src;
      bad |= !(r0 > 0.0f) || !(praw > 0.0f) || !isfinite(praw + (m1 + m2 + m3));
      const float p = vmax(praw, float(kPFloor));
      const float c = sqrtf((gamma * p) / rho);
      const float s = vmax(fabsf(u), vmax(fabsf(vv), fabsf(w))) + c;
      mn = fminf(mn, dx / s);
      two_sum_acc(hi[0], lo[0], r0);
      two_sum_acc(hi[1], lo[1], m1);
      two_sum_acc(hi[2], lo[2], m2);
      two_sum_acc(hi[3], lo[3], m3);
      two_sum_acc(hi[4], lo[4], E);
    }
  }
  double v[6];
  v[0] = double(mn);
#pragma unroll
  for (int k = 0; k < 5; ++k) v[k + 1] = double(hi[k]) + double(lo[k]);
  bad = __syncthreads_or(bad);
  block_reduce6(v, sh);
  if (threadIdx.x == 0) {
    const double dxd = ldexp(m.dx0, -lf.x);
    const double vol = dxd * dxd * dxd;
    partials[leaf * 6 + 0] = v[0];
    for (int k = 1; k < 6; ++k) partials[leaf * 6 + k] = v[k] * vol;
    if (bad && m.err) atomicOr(m.err, 1u);
  }
  __syncthreads();   // sh is rewritten by the next leaf
  }
}

#ifdef CELLO_DEFINE_FINISH_KERNEL
__global__ void __launch_bounds__(1024) reduce_finish_kernel(const double* partials, int B, double cfl,
                                                             double* dt_next, double* totals) {
  __shared__ double sh[6 * 32];
  double v[6] = {INFINITY, 0, 0, 0, 0, 0};
  for (int i = threadIdx.x; i < B; i += blockDim.x) {
    v[0] = fmin(v[0], partials[i * 6]);
    for (int k = 1; k < 6; ++k) v[k] += partials[i * 6 + k];
  }
  block_reduce6(v, sh);
  if (threadIdx.x == 0) {
    if (dt_next) *dt_next = cfl * v[0];
    if (totals)
      for (int k = 0; k < 5; ++k) totals[k] = v[k + 1];
  }
}
#endif

// =====================================================================
// Refinement flags: relative slope of rho or p, compared in float64.
// =====================================================================
template <typename T, int NB, int NF = 5>
__global__ void __launch_bounds__(256) flags_kernel(DevMesh m, const T* U, int field, double thr, double thr_c,
                                                    int8_t* flags) {
  constexpr int G = kGhosts, N = NB + 2 * G;
  constexpr long SLAB = (long)N * N * N;
  const int leaf = blockIdx.x;
  const int4 lf = m.leaf[leaf];
  const T* b = U + (long)leaf * NF * SLAB;
  const double gm1 = m.gamma - 1.0;
  auto q = [&](long o) -> double {
    const double r0 = double(b[o]);
    const double rho = r0 > kRhoFloor ? r0 : kRhoFloor;
    if (field == 0) return rho;
    const double u = double(b[SLAB + o]) / rho, v = double(b[2 * SLAB + o]) / rho, w = double(b[3 * SLAB + o]) / rho;
    const double ke = (0.5 * rho) * (u * u + (v * v + w * w));
    const double E = double(b[4 * SLAB + o]);
    double src = E - ke;
    if constexpr (NF == 6) src = (src > kDualEta1 * E) ? src : double(b[5 * SLAB + o]);
    const double p = gm1 * src;
    return p > kPFloor ? p : kPFloor;
  };
  int hit = 0, hit_c = 0;
  for (int i = threadIdx.x; i < NB * NB * NB; i += blockDim.x) {
    const int x = i % NB + G, y = (i / NB) % NB + G, z = i / (NB * NB) + G;
    const long o = ((long)z * N + y) * N + x;
    const double c = fabs(q(o));
    const long st[3] = {1, N, (long)N * N};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double diff = fabs(q(o + st[a]) - q(o - st[a]));
      hit |= diff > thr * c;
      hit_c |= diff > thr_c * c;
    }
  }
  hit = __syncthreads_or(hit);
  hit_c = __syncthreads_or(hit_c);
  if (threadIdx.x == 0) {
    int8_t f = 0;
    if (!hit_c && lf.x > 0) f = -1;
    if (hit && lf.x < m.max_level) f = 1;
    flags[leaf] = f;
  }
}

// =====================================================================
// Coarse-fine flux correction: one CTA per coarse leaf, its faces in order
// -x, +x, -y, +y, -z, +z, arithmetic in float64.
// =====================================================================
template <typename T, int NB, int NF = 5>
__global__ void __launch_bounds__(256) fluxcorr_kernel(DevMesh m, T* U, const CoarseFace* faces,
                                                       const int* group_start, const double* reg,
                                                       const double* dt) {
  constexpr int G = kGhosts, N = NB + 2 * G, H = NB / 2;
  constexpr long SLAB = (long)N * N * N;
  constexpr long FS = (long)NB * NB;
  const int f0 = group_start[blockIdx.x], f1 = group_start[blockIdx.x + 1];
  for (int fi = f0; fi < f1; ++fi) {
    const CoarseFace cf = faces[fi];
    const int4 cl = m.leaf[cf.leaf];
    const double dtdx = *dt / ldexp(m.dx0, -cl.x);
    const int t1a = cf.axis == 0 ? 1 : 0, t2a = cf.axis == 2 ? 1 : 2;
    for (int i = threadIdx.x; i < NB * NB; i += blockDim.x) {
      const int t1 = i % NB, t2 = i / NB;
      const int o1 = t1 / H, o2 = t2 / H;
      const int b1 = t1 - o1 * H, b2 = t2 - o2 * H;
      const double* Rf = reg + (long)cf.fslot[o2 * 2 + o1] * NF * FS + (2 * b2) * NB + 2 * b1;
      const double* Rc = reg + (long)cf.cslot * NF * FS + t2 * NB + t1;
      int cc[3];
      cc[cf.axis] = cf.side > 0 ? G + NB - 1 : G;
      cc[t1a] = G + t1;
      cc[t2a] = G + t2;
      T* cell = U + (long)cf.leaf * NF * SLAB + ((long)cc[2] * N + cc[1]) * N + cc[0];
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const double* r = Rf + f * FS;
        const double mean = ((r[0] + r[1]) + (r[NB] + r[NB + 1])) * 0.25;
        const double corr = (dtdx * (Rc[f * FS] - mean)) * double(cf.side);
        cell[f * SLAB] = T(double(cell[f * SLAB]) + corr);
      }
    }
    __syncthreads();
  }
}

}  // namespace cello
