// Multigrid Poisson solver (Sec. II.C: Enzo-P's mg0, a geometric multigrid
// V-cycle, the self-gravity solver of the paper's uniform-grid runs).  On a
// uniform periodic mesh the leaf interiors form one M^3 grid; the solver
// gathers them into one array in HBM, runs V-cycles on it and on its
// coarsenings (one array per level, periodic indexing, no ghost exchange:
// on one GPU the block decomposition has no reason to survive the gather),
// and scatters the result back to the leaves.  float64, no contraction.
//
// V-cycle (spacing h): two damped Jacobi sweeps (w = 6/7), the residual of
// the 8 children of each coarse cell restricted by their mean, a V-cycle for
// the coarse error from zero with spacing 2h, its trilinear prolongation
// added, two more sweeps; a 1-cell grid gives 0, an odd grid above 1 takes
// 50 sweeps.  Mean of f removed first, mean of phi removed last.
#include <vector>

#include "cello_internal.h"

namespace cello {
namespace {

constexpr double kOmega = 6.0 / 7.0;
constexpr int kNu = 2;
constexpr int kCoarseSweeps = 50;
constexpr int kRedThreads = 256;

// M <= 1024 (checked by cello_poisson_solve): M^3 <= 2^30 and every grid
// offset fits 32-bit unsigned arithmetic.
__device__ __forceinline__ unsigned gidx(int x, int y, int z, int M) {
  return ((unsigned)z * (unsigned)M + (unsigned)y) * (unsigned)M + (unsigned)x;
}
__device__ __forceinline__ int wrapm(int v, int M) { return v < 0 ? v + M : (v >= M ? v - M : v); }

template <typename T>
__device__ __forceinline__ T nbsum(const T* p, int x, int y, int z, int M) {
  const T xm = p[gidx(wrapm(x - 1, M), y, z, M)], xp = p[gidx(wrapm(x + 1, M), y, z, M)];
  const T ym = p[gidx(x, wrapm(y - 1, M), z, M)], yp = p[gidx(x, wrapm(y + 1, M), z, M)];
  const T zm = p[gidx(x, y, wrapm(z - 1, M), M)], zp = p[gidx(x, y, wrapm(z + 1, M), M)];
  return ((((xm + xp) + ym) + yp) + zm) + zp;
}

// The grid kernels run one thread per cell of an M^3 (or, for the
// restriction, (M/2)^3) grid on a 3-D launch: 32 x 8 threads per CTA in
// (x, y), one CTA row per z plane, so no division recovers the coordinates.
// The Jacobi sweep instead walks kZC planes per thread along z, keeping the
// z-1, z and z+1 values of its column in registers.
constexpr int kBX = 32, kBY = 8, kZC = 8;
dim3 grid3(int M) { return dim3((unsigned)((M + kBX - 1) / kBX), (unsigned)((M + kBY - 1) / kBY), (unsigned)M); }
dim3 grid_zc(int M) {
  return dim3((unsigned)((M + kBX - 1) / kBX), (unsigned)((M + kBY - 1) / kBY), (unsigned)((M + kZC - 1) / kZC));
}
const dim3 kBlock3(kBX, kBY, 1);

__device__ __forceinline__ bool cell3(int M, int& x, int& y, int& z) {
  x = blockIdx.x * kBX + threadIdx.x;
  y = blockIdx.y * kBY + threadIdx.y;
  z = blockIdx.z;
  return x < M && y < M;
}

template <typename T>
__global__ void jacobi_kernel(const T* __restrict__ in, T* __restrict__ out, const T* __restrict__ f, int M, T h2) {
  const int x = blockIdx.x * kBX + threadIdx.x;
  const int y = blockIdx.y * kBY + threadIdx.y;
  if (x >= M || y >= M) return;
  const int z0 = blockIdx.z * kZC;
  const int z1 = z0 + kZC < M ? z0 + kZC : M;
  const unsigned uM = (unsigned)M, P = uM * uM;
  const unsigned xm = (unsigned)wrapm(x - 1, M), xp = (unsigned)wrapm(x + 1, M);
  const unsigned row = (unsigned)y * uM, rym = (unsigned)wrapm(y - 1, M) * uM, ryp = (unsigned)wrapm(y + 1, M) * uM;
  unsigned zb = (unsigned)z0 * P;
  T cm = in[(unsigned)wrapm(z0 - 1, M) * P + row + x];   // column values at z-1 and z
  T cc = in[zb + row + x];
  for (int z = z0; z < z1; ++z) {
    const T cp = in[(unsigned)wrapm(z + 1, M) * P + row + x];
    // the neighbour sum in the order of nbsum: x-1, x+1, y-1, y+1, z-1, z+1
    const T s = ((((in[zb + row + xm] + in[zb + row + xp]) + in[zb + rym + x]) + in[zb + ryp + x]) + cm) + cp;
    const unsigned i = zb + row + x;
    out[i] = T(1.0 - kOmega) * cc + T(kOmega) * ((s - h2 * f[i]) * T(1.0 / 6.0));
    cm = cc;
    cc = cp;
    zb += P;
  }
}

// Coarse right-hand side: mean of the residuals f - lap(phi) of the 8
// children, in (dz, dy, dx) order.
template <typename T>
__global__ void residual_restrict_kernel(const T* __restrict__ phi, const T* __restrict__ f, T* __restrict__ fc,
                                         int M, T ih2) {
  const int Mc = M / 2;
  int X, Y, Z;
  if (!cell3(Mc, X, Y, Z)) return;
  const unsigned i = gidx(X, Y, Z, Mc);
  T s = T(0);
  bool first = true;
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        const int x = 2 * X + dx, y = 2 * Y + dy, z = 2 * Z + dz;
        const unsigned o = gidx(x, y, z, M);
        const T r = f[o] - (nbsum(phi, x, y, z, M) - T(6) * phi[o]) * ih2;
        s = first ? r : s + r;
        first = false;
      }
  fc[i] = s * T(0.125);
}

// phi += trilinear prolongation of the coarse error ec.
template <typename T>
__global__ void prolong_add_kernel(const T* __restrict__ ec, T* __restrict__ phi, int M) {
  const int Mc = M / 2;
  int x, y, z;
  if (!cell3(M, x, y, z)) return;
  const unsigned i = gidx(x, y, z, M);
  const int X = x >> 1, Y = y >> 1, Z = z >> 1;
  const int sx = (x & 1) ? 1 : -1, sy = (y & 1) ? 1 : -1, sz = (z & 1) ? 1 : -1;
  const int X1 = wrapm(X + sx, Mc), Y1 = wrapm(Y + sy, Mc), Z1 = wrapm(Z + sz, Mc);
  const T a = T(0.75), q = T(0.25);
  const T c00 = a * ec[gidx(X, Y, Z, Mc)] + q * ec[gidx(X1, Y, Z, Mc)];
  const T c10 = a * ec[gidx(X, Y1, Z, Mc)] + q * ec[gidx(X1, Y1, Z, Mc)];
  const T c01 = a * ec[gidx(X, Y, Z1, Mc)] + q * ec[gidx(X1, Y, Z1, Mc)];
  const T c11 = a * ec[gidx(X, Y1, Z1, Mc)] + q * ec[gidx(X1, Y1, Z1, Mc)];
  const T c0 = a * c00 + q * c10;
  const T c1 = a * c01 + q * c11;
  phi[i] = phi[i] + (a * c0 + q * c1);
}

// Mixed precision: the float64 residual rounded to float32 (the right-hand
// side of a float32 V-cycle), and the float32 correction added to phi.
__global__ void residual_f32_kernel(const double* __restrict__ phi, const double* __restrict__ f,
                                    float* __restrict__ r, int M, double ih2) {
  int x, y, z;
  if (!cell3(M, x, y, z)) return;
  const unsigned i = gidx(x, y, z, M);
  r[i] = (float)(f[i] - (nbsum(phi, x, y, z, M) - 6.0 * phi[i]) * ih2);
}

__global__ void correct_kernel(double* __restrict__ phi, const float* __restrict__ e, long count) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) phi[i] = phi[i] + (double)e[i];
}

template <typename T>
__global__ void fill_kernel(T* p, long count, T v) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) p[i] = v;
}

__global__ void add_kernel(double* p, long count, const double* shift, double scale) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) p[i] = p[i] - *shift * scale;
}

// Partial sums (op 0) or max |residual| (op 1) per CTA, then one CTA folds them.
__global__ void reduce_kernel(const double* __restrict__ a, const double* __restrict__ f, long count, int M,
                              double ih2, int op, double* __restrict__ partial) {
  __shared__ double sh[kRedThreads];
  double acc = 0.0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x) {
    if (op == 0) {
      acc += a[i];
    } else {
      const unsigned u = (unsigned)i, uM = (unsigned)M;   // M^3 <= 2^30: 32-bit index arithmetic
      const int x = (int)(u % uM), y = (int)((u / uM) % uM), z = (int)(u / (uM * uM));
      const double r = fabs(f[i] - (nbsum(a, x, y, z, M) - 6.0 * a[i]) * ih2);
      acc = r > acc ? r : acc;
    }
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kRedThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      const double o = sh[threadIdx.x + s];
      sh[threadIdx.x] = op == 0 ? sh[threadIdx.x] + o : (o > sh[threadIdx.x] ? o : sh[threadIdx.x]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void fold_kernel(const double* __restrict__ partial, int n, int op, double scale, double* out) {
  __shared__ double sh[kRedThreads];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc = op == 0 ? acc + partial[i] : fmax(acc, partial[i]);
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kRedThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      sh[threadIdx.x] = op == 0 ? sh[threadIdx.x] + sh[threadIdx.x + s] : fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0] * scale;
}

// Leaf interiors [B][n^3] <-> the global grid (to_global = 1 gathers).
__global__ void leaves_grid_kernel(const int4* leaf, int B, int n, int M, double* leaves, double* grid, int to_global) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long n3 = (long)n * n * n;
  if (i >= (long)B * n3) return;
  const int b = (int)(i / n3);
  const int c = (int)(i - (long)b * n3);
  const int x = c % n, y = (c / n) % n, z = c / (n * n);
  const int4 lf = leaf[b];
  const long g = gidx(lf.y * n + x, lf.z * n + y, lf.w * n + z, M);
  if (to_global) grid[g] = leaves[i];
  else leaves[i] = grid[g];
}

unsigned blocks_for(long count) { return (unsigned)((count + 255) / 256); }

template <typename T>
struct Level {
  int M;
  double h;
  T *phi, *tmp, *f;
};

template <typename T>
struct Cycle {
  std::vector<Level<T>> lv;
  cudaStream_t s;

  void sweeps(Level<T>& L, int count) {
    for (int k = 0; k < count; ++k) {
      jacobi_kernel<T><<<grid_zc(L.M), kBlock3, 0, s>>>(L.phi, L.tmp, L.f, L.M, T(L.h * L.h));
      std::swap(L.phi, L.tmp);
    }
  }

  void vcycle(int l) {
    Level<T>& L = lv[l];
    if (L.M == 1) {
      fill_kernel<T><<<1, 32, 0, s>>>(L.phi, 1, T(0));
      return;
    }
    if (L.M % 2 == 1) {
      sweeps(L, kCoarseSweeps);
      return;
    }
    sweeps(L, kNu);
    Level<T>& C = lv[l + 1];
    const long cc = (long)C.M * C.M * C.M;
    residual_restrict_kernel<T><<<grid3(C.M), kBlock3, 0, s>>>(L.phi, L.f, C.f, L.M, T(1.0 / (L.h * L.h)));
    fill_kernel<T><<<blocks_for(cc), 256, 0, s>>>(C.phi, cc, T(0));
    vcycle(l + 1);
    prolong_add_kernel<T><<<grid3(L.M), kBlock3, 0, s>>>(C.phi, L.phi, L.M);
    sweeps(L, kNu);
  }
};

}  // namespace

// Scratch of the solver for one mesh: the level arrays (float64 and, for
// mixed precision, float32), the reduction partials.  Allocated on the
// first solve of each kind, freed with the mesh.
struct PoissonScratch {
  std::vector<void*> d64, d32;
  double* red = nullptr;   // 1024 partials + 2 scalars
  ~PoissonScratch() {
    for (void* p : d64) cudaFree(p);
    for (void* p : d32) cudaFree(p);
    if (red) cudaFree(red);
  }
};

void poisson_free(PoissonScratch* p) { delete p; }

namespace {

// Three arrays per level, for the levels not yet allocated.
cudaError_t alloc_levels(std::vector<void*>& bufs, const std::vector<int>& sizes, size_t elem) {
  for (size_t l = bufs.size() / 3; l < sizes.size(); ++l)
    for (int k = 0; k < 3; ++k) {
      const int Ml = sizes[l];
      void* d = nullptr;
      cudaError_t e = cudaMalloc(&d, elem * (size_t)Ml * Ml * Ml);
      if (e != cudaSuccess) return e;
      bufs.push_back(d);
    }
  return cudaSuccess;
}

template <typename T>
Cycle<T> make_cycle(const std::vector<void*>& bufs, const std::vector<int>& sizes, double h, cudaStream_t s) {
  Cycle<T> C;
  C.s = s;
  for (size_t l = 0; l < sizes.size(); ++l)
    C.lv.push_back(Level<T>{sizes[l], h * (double)(1L << l), static_cast<T*>(bufs[3 * l]),
                            static_cast<T*>(bufs[3 * l + 1]), static_cast<T*>(bufs[3 * l + 2])});
  return C;
}

// scalar = mean of a (op 0) or max |f - lap(a)| (op 1) on the finest grid
void reduce_to(const double* a, const double* f, int M, double h, int op, double* red, double* out, cudaStream_t s) {
  const long c = (long)M * M * M;
  reduce_kernel<<<1024, kRedThreads, 0, s>>>(a, f, c, M, 1.0 / (h * h), op, red);
  fold_kernel<<<1, kRedThreads, 0, s>>>(red, 1024, op, op == 0 ? 1.0 / (double)c : 1.0, out);
}

}  // namespace

cudaError_t poisson_solve(PoissonScratch** scratch, const DevMesh& m, int M, double h, const double* f_leaves,
                          double* phi_leaves, int cycles, int inner, double* resid_host, cudaStream_t s) {
  std::vector<int> sizes;
  for (int Ml = M;; Ml /= 2) {
    sizes.push_back(Ml);
    if (Ml == 1 || Ml % 2 == 1) break;
  }
  if (!*scratch) *scratch = new PoissonScratch();
  PoissonScratch* P = *scratch;
  cudaError_t e = alloc_levels(P->d64, inner == 8 ? sizes : std::vector<int>{M}, sizeof(double));
  if (e == cudaSuccess && inner == 4) e = alloc_levels(P->d32, sizes, sizeof(float));
  if (e == cudaSuccess && !P->red) e = cudaMalloc(&P->red, sizeof(double) * (1024 + 2));
  if (e != cudaSuccess) return e;
  double* scalar = P->red + 1024;
  // the float64 finest grid: level 0 of the float64 hierarchy
  double* phi = static_cast<double*>(P->d64[0]);
  double* tmp = static_cast<double*>(P->d64[1]);
  double* f = static_cast<double*>(P->d64[2]);
  const long c = (long)M * M * M;
  const long nl = (long)m.B * m.n * m.n * m.n;
  leaves_grid_kernel<<<blocks_for(nl), 256, 0, s>>>(m.leaf, m.B, m.n, M, const_cast<double*>(f_leaves), f, 1);
  reduce_to(f, nullptr, M, h, 0, P->red, scalar, s);
  add_kernel<<<blocks_for(c), 256, 0, s>>>(f, c, scalar, 1.0);
  fill_kernel<double><<<blocks_for(c), 256, 0, s>>>(phi, c, 0.0);
  Cycle<double> C64;
  Cycle<float> C32;
  if (inner == 8) C64 = make_cycle<double>(P->d64, sizes, h, s);
  else C32 = make_cycle<float>(P->d32, sizes, h, s);
  for (int k = 0; k < cycles; ++k) {
    if (inner == 8) {
      C64.vcycle(0);
    } else {
      Level<float>& L = C32.lv[0];
      residual_f32_kernel<<<grid3(M), kBlock3, 0, s>>>(phi, f, L.f, M, 1.0 / (h * h));
      fill_kernel<float><<<blocks_for(c), 256, 0, s>>>(L.phi, c, 0.0f);
      C32.vcycle(0);
      correct_kernel<<<blocks_for(c), 256, 0, s>>>(phi, L.phi, c);
    }
    const double* cur = inner == 8 ? C64.lv[0].phi : phi;
    if (resid_host) {
      reduce_to(cur, f, M, h, 1, P->red, scalar + 1, s);
      e = cudaMemcpyAsync(resid_host + k, scalar + 1, sizeof(double), cudaMemcpyDeviceToHost, s);
      if (e != cudaSuccess) return e;
    }
  }
  double* out = inner == 8 ? C64.lv[0].phi : phi;
  (void)tmp;
  reduce_to(out, nullptr, M, h, 0, P->red, scalar, s);
  add_kernel<<<blocks_for(c), 256, 0, s>>>(out, c, scalar, 1.0);
  leaves_grid_kernel<<<blocks_for(nl), 256, 0, s>>>(m.leaf, m.B, m.n, M, phi_leaves, out, 0);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (resid_host) e = cudaStreamSynchronize(s);
  return e;
}

}  // namespace cello
