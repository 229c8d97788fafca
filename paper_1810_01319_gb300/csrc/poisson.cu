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

__device__ __forceinline__ long gidx(int x, int y, int z, int M) { return ((long)z * M + y) * M + x; }
__device__ __forceinline__ int wrapm(int v, int M) { return v < 0 ? v + M : (v >= M ? v - M : v); }

__device__ __forceinline__ double nbsum(const double* p, int x, int y, int z, int M) {
  const double xm = p[gidx(wrapm(x - 1, M), y, z, M)], xp = p[gidx(wrapm(x + 1, M), y, z, M)];
  const double ym = p[gidx(x, wrapm(y - 1, M), z, M)], yp = p[gidx(x, wrapm(y + 1, M), z, M)];
  const double zm = p[gidx(x, y, wrapm(z - 1, M), M)], zp = p[gidx(x, y, wrapm(z + 1, M), M)];
  return ((((xm + xp) + ym) + yp) + zm) + zp;
}

__global__ void jacobi_kernel(const double* __restrict__ in, double* __restrict__ out, const double* __restrict__ f,
                              int M, double h2) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)M * M * M) return;
  const unsigned u = (unsigned)i, uM = (unsigned)M;   // M^3 <= 2^30: 32-bit index arithmetic
  const int x = (int)(u % uM), y = (int)((u / uM) % uM), z = (int)(u / (uM * uM));
  out[i] = (1.0 - kOmega) * in[i] + kOmega * ((nbsum(in, x, y, z, M) - h2 * f[i]) * (1.0 / 6.0));
}

// Coarse right-hand side: mean of the residuals f - lap(phi) of the 8
// children, in (dz, dy, dx) order.
__global__ void residual_restrict_kernel(const double* __restrict__ phi, const double* __restrict__ f,
                                         double* __restrict__ fc, int M, double ih2) {
  const int Mc = M / 2;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)Mc * Mc * Mc) return;
  const unsigned u = (unsigned)i, uM = (unsigned)Mc;
  const int X = (int)(u % uM), Y = (int)((u / uM) % uM), Z = (int)(u / (uM * uM));
  double s = 0.0;
  bool first = true;
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        const int x = 2 * X + dx, y = 2 * Y + dy, z = 2 * Z + dz;
        const long o = gidx(x, y, z, M);
        const double r = f[o] - (nbsum(phi, x, y, z, M) - 6.0 * phi[o]) * ih2;
        s = first ? r : s + r;
        first = false;
      }
  fc[i] = s * 0.125;
}

// phi += trilinear prolongation of the coarse error ec.
__global__ void prolong_add_kernel(const double* __restrict__ ec, double* __restrict__ phi, int M) {
  const int Mc = M / 2;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)M * M * M) return;
  const unsigned u = (unsigned)i, uM = (unsigned)M;   // M^3 <= 2^30: 32-bit index arithmetic
  const int x = (int)(u % uM), y = (int)((u / uM) % uM), z = (int)(u / (uM * uM));
  const int X = x >> 1, Y = y >> 1, Z = z >> 1;
  const int sx = (x & 1) ? 1 : -1, sy = (y & 1) ? 1 : -1, sz = (z & 1) ? 1 : -1;
  const int X1 = wrapm(X + sx, Mc), Y1 = wrapm(Y + sy, Mc), Z1 = wrapm(Z + sz, Mc);
  const double c00 = 0.75 * ec[gidx(X, Y, Z, Mc)] + 0.25 * ec[gidx(X1, Y, Z, Mc)];
  const double c10 = 0.75 * ec[gidx(X, Y1, Z, Mc)] + 0.25 * ec[gidx(X1, Y1, Z, Mc)];
  const double c01 = 0.75 * ec[gidx(X, Y, Z1, Mc)] + 0.25 * ec[gidx(X1, Y, Z1, Mc)];
  const double c11 = 0.75 * ec[gidx(X, Y1, Z1, Mc)] + 0.25 * ec[gidx(X1, Y1, Z1, Mc)];
  const double c0 = 0.75 * c00 + 0.25 * c10;
  const double c1 = 0.75 * c01 + 0.25 * c11;
  phi[i] = phi[i] + (0.75 * c0 + 0.25 * c1);
}

__global__ void fill_kernel(double* p, long count, double v) {
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

struct Level {
  int M;
  double h;
  double *phi, *tmp, *f;
};

struct Solver {
  std::vector<Level> lv;
  double* partial;
  int npart;
  double* scalar;   // [2]: mean, residual max
  cudaStream_t s;

  void sweeps(Level& L, int count) {
    const long c = (long)L.M * L.M * L.M;
    for (int k = 0; k < count; ++k) {
      jacobi_kernel<<<blocks_for(c), 256, 0, s>>>(L.phi, L.tmp, L.f, L.M, L.h * L.h);
      std::swap(L.phi, L.tmp);
    }
  }

  void vcycle(int l) {
    Level& L = lv[l];
    const long c = (long)L.M * L.M * L.M;
    if (L.M == 1) {
      fill_kernel<<<1, 32, 0, s>>>(L.phi, 1, 0.0);
      return;
    }
    if (L.M % 2 == 1) {
      sweeps(L, kCoarseSweeps);
      return;
    }
    sweeps(L, kNu);
    Level& C = lv[l + 1];
    const long cc = (long)C.M * C.M * C.M;
    residual_restrict_kernel<<<blocks_for(cc), 256, 0, s>>>(L.phi, L.f, C.f, L.M, 1.0 / (L.h * L.h));
    fill_kernel<<<blocks_for(cc), 256, 0, s>>>(C.phi, cc, 0.0);
    vcycle(l + 1);
    prolong_add_kernel<<<blocks_for(c), 256, 0, s>>>(C.phi, L.phi, L.M);
    sweeps(L, kNu);
  }

  // scalar[slot] = mean of a (op 0) or max |f - lap(a)| (op 1) on level 0
  void reduce(const double* a, const double* f, int op, int slot) {
    const Level& L = lv[0];
    const long c = (long)L.M * L.M * L.M;
    reduce_kernel<<<npart, kRedThreads, 0, s>>>(a, f, c, L.M, 1.0 / (L.h * L.h), op, partial);
    fold_kernel<<<1, kRedThreads, 0, s>>>(partial, npart, op, op == 0 ? 1.0 / (double)c : 1.0, scalar + slot);
  }
};

}  // namespace

// Scratch of the solver for one mesh: the level arrays, the reduction
// partials.  Allocated on the first solve, freed with the mesh.
struct PoissonScratch {
  std::vector<double*> bufs;
  ~PoissonScratch() {
    for (double* p : bufs) cudaFree(p);
  }
};

void poisson_free(PoissonScratch* p) { delete p; }

cudaError_t poisson_solve(PoissonScratch** scratch, const DevMesh& m, int M, double h, const double* f_leaves,
                          double* phi_leaves, int cycles, double* resid_host, cudaStream_t s) {
  std::vector<int> sizes;
  for (int Ml = M;; Ml /= 2) {
    sizes.push_back(Ml);
    if (Ml == 1 || Ml % 2 == 1) break;
  }
  if (!*scratch) {
    auto* p = new PoissonScratch();
    for (int Ml : sizes) {
      const size_t bytes = sizeof(double) * (size_t)Ml * Ml * Ml;
      for (int k = 0; k < 3; ++k) {
        double* d = nullptr;
        cudaError_t e = cudaMalloc(&d, bytes);
        if (e != cudaSuccess) {
          delete p;
          return e;
        }
        p->bufs.push_back(d);
      }
    }
    double* d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(double) * (1024 + 2));
    if (e != cudaSuccess) {
      delete p;
      return e;
    }
    p->bufs.push_back(d);
    *scratch = p;
  }
  Solver S;
  S.s = s;
  for (size_t l = 0; l < sizes.size(); ++l)
    S.lv.push_back(Level{sizes[l], h * (double)(1L << l), (*scratch)->bufs[3 * l], (*scratch)->bufs[3 * l + 1],
                         (*scratch)->bufs[3 * l + 2]});
  S.partial = (*scratch)->bufs.back();
  S.npart = 1024;
  S.scalar = S.partial + 1024;
  Level& L0 = S.lv[0];
  const long c = (long)M * M * M;
  const long nl = (long)m.B * m.n * m.n * m.n;
  leaves_grid_kernel<<<blocks_for(nl), 256, 0, s>>>(m.leaf, m.B, m.n, M, const_cast<double*>(f_leaves), L0.f, 1);
  S.reduce(L0.f, nullptr, 0, 0);
  add_kernel<<<blocks_for(c), 256, 0, s>>>(L0.f, c, S.scalar, 1.0);
  fill_kernel<<<blocks_for(c), 256, 0, s>>>(L0.phi, c, 0.0);
  for (int k = 0; k < cycles; ++k) {
    S.vcycle(0);
    if (resid_host) {
      S.reduce(L0.phi, L0.f, 1, 1);
      cudaError_t e = cudaMemcpyAsync(resid_host + k, S.scalar + 1, sizeof(double), cudaMemcpyDeviceToHost, s);
      if (e != cudaSuccess) return e;
    }
  }
  S.reduce(L0.phi, nullptr, 0, 0);
  add_kernel<<<blocks_for(c), 256, 0, s>>>(L0.phi, c, S.scalar, 1.0);
  leaves_grid_kernel<<<blocks_for(nl), 256, 0, s>>>(m.leaf, m.B, m.n, M, phi_leaves, L0.phi, 0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (resid_host) e = cudaStreamSynchronize(s);
  return e;
}

}  // namespace cello
