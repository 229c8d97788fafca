// Multigrid Poisson solver (Sec. II.C: Enzo-P's mg0, a geometric multigrid
// V-cycle, the self-gravity solver of the paper's uniform-grid runs) on the
// block table of a uniform periodic mesh.
//
// Each leaf block carries its own grid on every level where a block still
// has at least 4 cells per edge (n, n/2, ..., 4), as an array of padded
// blocks [B][(n_l + 2)^3] with a one-cell ghost layer.  Before every stencil
// the ghost layer is refreshed from the same-level neighbour blocks through
// the 27-entry neighbour table of the hydro refresh (every ghost cell takes
// the interior cell of the neighbour leaf in its direction; the periodic
// wrap is in the table).  Below the last block level the restricted
// residual of the blocks forms one grid of 2 cells per block edge, and the
// remaining coarse levels are single arrays with periodic indexing (a block
// of one or two cells has nothing left to exchange that the index wrap does
// not already give).  float64, no contraction.
//
// V-cycle (spacing h): two damped Jacobi sweeps (w = 6/7), the residual of
// the 8 children of each coarse cell restricted by their mean, a V-cycle for
// the coarse error from zero with spacing 2h, its trilinear prolongation
// added, two more sweeps; a 1-cell grid gives 0, an odd grid above 1 takes
// 50 sweeps.  Mean of f removed first, mean of phi removed last.  Every value
// is the oracle's expression in its order on the same grid values (the
// block layout only changes where they are stored); the Laplacian's 1/h^2
// and the Jacobi 1/6 are multiplications by reciprocals computed once.
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

// ---------------------------------------------------------------------------
// Block levels: arrays of padded blocks [B][P^3], P = n + 2 (one ghost cell),
// interior cells at padded coordinates 1 .. n.
__device__ __forceinline__ long bidx(int b, int x, int y, int z, int P) {
  return (((long)b * P + z) * P + y) * P + x;
}

// Block edges are powers of two (n, n/2, ..., 4): global cell gid of a
// level -> block b and padded coordinates of its interior cell (x fastest),
// by shifts and masks.
__device__ __forceinline__ int blk_cell(long gid, int n, int& x, int& y, int& z) {
  const int ln = __ffs(n) - 1;
  const int c = (int)(gid & (((long)1 << (3 * ln)) - 1));
  x = (c & (n - 1)) + 1;
  y = ((c >> ln) & (n - 1)) + 1;
  z = (c >> (2 * ln)) + 1;
  return (int)(gid >> (3 * ln));
}

// Ghost layer of every block: each ghost cell takes the interior cell of the
// same-level neighbour leaf in its direction (the 27-entry table; the mesh
// is uniform and periodic, so every entry is a same-level leaf).  Ghost cell
// q of a block: the z planes 0 and P-1, then the y rows 0 and P-1 of the
// interior z planes, then the x columns 0 and P-1 of the interior rows.
template <typename T>
__global__ void blk_refresh_kernel(DevMesh m, T* a, int n, int B) {
  const int P = n + 2;
  const long per = (long)P * P * P - (long)n * n * n;
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long)B * per) return;
  const int b = (int)(gid / per);
  int q = (int)(gid - (long)b * per);
  int x, y, z;
  if (q < 2 * P * P) {
    z = q < P * P ? 0 : P - 1;
    q %= P * P;
    y = q / P;
    x = q % P;
  } else if (q < 2 * P * P + 2 * n * P) {
    q -= 2 * P * P;
    z = 1 + q / (2 * P);
    const int r = q % (2 * P);
    y = r < P ? 0 : P - 1;
    x = r % P;
  } else {
    q -= 2 * P * P + 2 * n * P;
    z = 1 + q / (2 * n);
    const int r = q % (2 * n);
    y = 1 + r / 2;
    x = (r & 1) ? P - 1 : 0;
  }
  const int d0 = x == 0 ? -1 : (x == P - 1 ? 1 : 0);
  const int d1 = y == 0 ? -1 : (y == P - 1 ? 1 : 0);
  const int d2 = z == 0 ? -1 : (z == P - 1 ? 1 : 0);
  const int src = m.idx[b * 27 + (d2 + 1) * 9 + (d1 + 1) * 3 + (d0 + 1)];
  a[bidx(b, x, y, z, P)] = a[bidx(src, x - d0 * n, y - d1 * n, z - d2 * n, P)];
}

template <typename T>
__device__ __forceinline__ T bnbsum(const T* p, long i, int P) {
  const long PP = (long)P * P;
  return ((((p[i - 1] + p[i + 1]) + p[i - P]) + p[i + P]) + p[i - PP]) + p[i + PP];
}

// Damped Jacobi sweep over every block's interior (ghosts of `in` refreshed).
template <typename T>
__global__ void blk_jacobi_kernel(const T* __restrict__ in, T* __restrict__ out, const T* __restrict__ f, int n,
                                  int B, T h2) {
  const long n3 = (long)n * n * n;
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long)B * n3) return;
  int x, y, z;
  const int b = blk_cell(gid, n, x, y, z);
  const int P = n + 2;
  const long i = bidx(b, x, y, z, P);
  out[i] = T(1.0 - kOmega) * in[i] + T(kOmega) * ((bnbsum(in, i, P) - h2 * f[i]) * T(1.0 / 6.0));
}

// Residual f - lap(phi) of the 8 children of each coarse cell, their mean in
// (dz, dy, dx) order: into the next block level (g == nullptr) or into the
// global grid of Mg cells per axis (coarse cell of block b at global
// (i n/2 + X, j n/2 + Y, k n/2 + Z)).
template <typename T>
__global__ void blk_residual_restrict_kernel(DevMesh m, const T* __restrict__ phi, const T* __restrict__ f,
                                             T* __restrict__ fc, T* __restrict__ g, int Mg, int n, int B, T ih2) {
  const int nc = n / 2, P = n + 2, Pc = nc + 2;
  const long nc3 = (long)nc * nc * nc;
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long)B * nc3) return;
  int X, Y, Z;
  const int b = blk_cell(gid, nc, X, Y, Z);   // padded: 1 .. nc
  T s = T(0);
  bool first = true;
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        const long o = bidx(b, 2 * X - 1 + dx, 2 * Y - 1 + dy, 2 * Z - 1 + dz, P);
        const T r = f[o] - (bnbsum(phi, o, P) - T(6) * phi[o]) * ih2;
        s = first ? r : s + r;
        first = false;
      }
  if (g) {
    const int4 lf = m.leaf[b];
    g[gidx(lf.y * nc + X - 1, lf.z * nc + Y - 1, lf.w * nc + Z - 1, Mg)] = s * T(0.125);
  } else {
    fc[bidx(b, X, Y, Z, Pc)] = s * T(0.125);
  }
}

// phi += trilinear prolongation of the coarse error: from the next block
// level ec (its ghosts refreshed, edges and corners included), or from the
// global grid g of Mc cells per axis (periodic indexing).
template <typename T>
__global__ void blk_prolong_add_kernel(DevMesh m, const T* __restrict__ ec, const T* __restrict__ g, int Mc,
                                       T* __restrict__ phi, int n, int B) {
  const long n3 = (long)n * n * n;
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long)B * n3) return;
  int x, y, z;
  const int b = blk_cell(gid, n, x, y, z);
  const int P = n + 2, nc = n / 2, Pc = nc + 2;
  // interior offsets 0 .. n-1; the parent and the nearer coarse neighbour
  const int ix = x - 1, iy = y - 1, iz = z - 1;
  const int sx = (ix & 1) ? 1 : -1, sy = (iy & 1) ? 1 : -1, sz = (iz & 1) ? 1 : -1;
  const T a = T(0.75), q = T(0.25);
  T e000, e100, e010, e110, e001, e101, e011, e111;
  if (g) {
    const int4 lf = m.leaf[b];
    const int X = (lf.y * n + ix) >> 1, Y = (lf.z * n + iy) >> 1, Z = (lf.w * n + iz) >> 1;
    const int X1 = wrapm(X + sx, Mc), Y1 = wrapm(Y + sy, Mc), Z1 = wrapm(Z + sz, Mc);
    e000 = g[gidx(X, Y, Z, Mc)]; e100 = g[gidx(X1, Y, Z, Mc)];
    e010 = g[gidx(X, Y1, Z, Mc)]; e110 = g[gidx(X1, Y1, Z, Mc)];
    e001 = g[gidx(X, Y, Z1, Mc)]; e101 = g[gidx(X1, Y, Z1, Mc)];
    e011 = g[gidx(X, Y1, Z1, Mc)]; e111 = g[gidx(X1, Y1, Z1, Mc)];
  } else {
    const int X = (ix >> 1) + 1, Y = (iy >> 1) + 1, Z = (iz >> 1) + 1;   // padded coarse coordinates
    const int X1 = X + sx, Y1 = Y + sy, Z1 = Z + sz;
    e000 = ec[bidx(b, X, Y, Z, Pc)]; e100 = ec[bidx(b, X1, Y, Z, Pc)];
    e010 = ec[bidx(b, X, Y1, Z, Pc)]; e110 = ec[bidx(b, X1, Y1, Z, Pc)];
    e001 = ec[bidx(b, X, Y, Z1, Pc)]; e101 = ec[bidx(b, X1, Y, Z1, Pc)];
    e011 = ec[bidx(b, X, Y1, Z1, Pc)]; e111 = ec[bidx(b, X1, Y1, Z1, Pc)];
  }
  const T c00 = a * e000 + q * e100;
  const T c10 = a * e010 + q * e110;
  const T c01 = a * e001 + q * e101;
  const T c11 = a * e011 + q * e111;
  const T c0 = a * c00 + q * c10;
  const T c1 = a * c01 + q * c11;
  const long i = bidx(b, x, y, z, P);
  phi[i] = phi[i] + (a * c0 + q * c1);
}

// Level 0 in and out: compact leaf interiors [B][n^3] <-> padded blocks.
// in: dst = src - *shift (the mean of f); out: dst = src.
__global__ void blk_from_leaves_kernel(const double* __restrict__ src, double* __restrict__ dst, int n, int B,
                                       const double* shift) {
  const long n3 = (long)n * n * n;
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long)B * n3) return;
  int x, y, z;
  const int b = blk_cell(gid, n, x, y, z);
  dst[bidx(b, x, y, z, n + 2)] = src[gid] - *shift;
}

__global__ void blk_to_leaves_kernel(const double* __restrict__ src, double* __restrict__ dst, int n, int B) {
  const long n3 = (long)n * n * n;
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long)B * n3) return;
  int x, y, z;
  const int b = blk_cell(gid, n, x, y, z);
  dst[gid] = src[bidx(b, x, y, z, n + 2)];
}

// Mixed precision on level 0: the float64 residual rounded to float32 (the
// right-hand side of a float32 V-cycle), and the float32 correction added.
__global__ void blk_residual_f32_kernel(const double* __restrict__ phi, const double* __restrict__ f,
                                        float* __restrict__ r, int n, int B, double ih2) {
  const long n3 = (long)n * n * n;
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long)B * n3) return;
  int x, y, z;
  const int b = blk_cell(gid, n, x, y, z);
  const long i = bidx(b, x, y, z, n + 2);
  r[i] = (float)(f[i] - (bnbsum(phi, i, n + 2) - 6.0 * phi[i]) * ih2);
}

__global__ void blk_correct_kernel(double* __restrict__ phi, const float* __restrict__ e, int n, int B) {
  const long n3 = (long)n * n * n;
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= (long)B * n3) return;
  int x, y, z;
  const int b = blk_cell(gid, n, x, y, z);
  const long i = bidx(b, x, y, z, n + 2);
  phi[i] = phi[i] + (double)e[i];
}

// max |f - lap(phi)| over the interiors (ghosts of phi refreshed): one
// partial per CTA.
__global__ void blk_resmax_kernel(const double* __restrict__ phi, const double* __restrict__ f, int n, int B,
                                  double ih2, double* __restrict__ partial) {
  __shared__ double sh[kRedThreads];
  const long n3 = (long)n * n * n, count = (long)B * n3;
  double acc = 0.0;
  for (long gid = (long)blockIdx.x * blockDim.x + threadIdx.x; gid < count; gid += (long)gridDim.x * blockDim.x) {
    int x, y, z;
    const int b = blk_cell(gid, n, x, y, z);
    const long i = bidx(b, x, y, z, n + 2);
    const double r = fabs(f[i] - (bnbsum(phi, i, n + 2) - 6.0 * phi[i]) * ih2);
    acc = r > acc ? r : acc;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kRedThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

unsigned blocks_for(long count) { return (unsigned)((count + 255) / 256); }

template <typename T>
struct Level {
  int M;
  double h;
  T *phi, *tmp, *f;
};

// The single-array coarse levels.
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

// A block level: n cells per block edge, spacing h, padded arrays.
template <typename T>
struct BLevel {
  int n;
  double h;
  T *phi, *tmp, *f;
};

// The V-cycle over the block levels, then the single-array tail.
template <typename T>
struct BlockCycle {
  DevMesh m;
  int B;
  std::vector<BLevel<T>> blk;
  Cycle<T> tail;
  cudaStream_t s;

  void refresh(const BLevel<T>& L, T* a) {
    const long g = (long)B * ((long)(L.n + 2) * (L.n + 2) * (L.n + 2) - (long)L.n * L.n * L.n);
    blk_refresh_kernel<T><<<blocks_for(g), 256, 0, s>>>(m, a, L.n, B);
  }

  void sweeps(BLevel<T>& L, int count) {
    const long c = (long)B * L.n * L.n * L.n;
    for (int k = 0; k < count; ++k) {
      refresh(L, L.phi);
      blk_jacobi_kernel<T><<<blocks_for(c), 256, 0, s>>>(L.phi, L.tmp, L.f, L.n, B, T(L.h * L.h));
      std::swap(L.phi, L.tmp);
    }
  }

  void vcycle(int l) {
    BLevel<T>& L = blk[l];
    sweeps(L, kNu);
    refresh(L, L.phi);
    const long cc = (long)B * (L.n / 2) * (L.n / 2) * (L.n / 2);
    const T ih2 = T(1.0 / (L.h * L.h));
    if (l + 1 < (int)blk.size()) {
      BLevel<T>& C = blk[l + 1];
      const long pc = (long)B * (C.n + 2) * (C.n + 2) * (C.n + 2);
      blk_residual_restrict_kernel<T><<<blocks_for(cc), 256, 0, s>>>(m, L.phi, L.f, C.f, nullptr, 0, L.n, B, ih2);
      fill_kernel<T><<<blocks_for(pc), 256, 0, s>>>(C.phi, pc, T(0));
      vcycle(l + 1);
      refresh(C, C.phi);
      blk_prolong_add_kernel<T><<<blocks_for((long)B * L.n * L.n * L.n), 256, 0, s>>>(m, C.phi, nullptr, 0, L.phi,
                                                                                    L.n, B);
    } else {
      Level<T>& G = tail.lv[0];
      const long gc = (long)G.M * G.M * G.M;
      blk_residual_restrict_kernel<T><<<blocks_for(cc), 256, 0, s>>>(m, L.phi, L.f, nullptr, G.f, G.M, L.n, B, ih2);
      fill_kernel<T><<<blocks_for(gc), 256, 0, s>>>(G.phi, gc, T(0));
      tail.vcycle(0);
      blk_prolong_add_kernel<T><<<blocks_for((long)B * L.n * L.n * L.n), 256, 0, s>>>(m, nullptr, G.phi, G.M,
                                                                                    L.phi, L.n, B);
    }
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

// Three arrays per level (cells per array given), for the levels not yet
// allocated.
cudaError_t alloc_levels(std::vector<void*>& bufs, const std::vector<long>& cells, size_t elem) {
  for (size_t l = bufs.size() / 3; l < cells.size(); ++l)
    for (int k = 0; k < 3; ++k) {
      void* d = nullptr;
      cudaError_t e = cudaMalloc(&d, elem * (size_t)cells[l]);
      if (e != cudaSuccess) return e;
      bufs.push_back(d);
    }
  return cudaSuccess;
}

// The level structure: block levels n, n/2, ..., 4, then single arrays of
// M = root 2^L 2 cells per axis, halved while even and above 1.
struct Plan {
  std::vector<int> bn;      // cells per block edge of the block levels
  std::vector<int> gm;      // cells per axis of the single-array levels
  std::vector<long> cells;  // cells of each level's arrays, block levels first
};

Plan plan_levels(int B, int n, int Mblocks) {
  Plan p;
  for (int nl = n; nl >= 4; nl /= 2) {
    p.bn.push_back(nl);
    p.cells.push_back((long)B * (nl + 2) * (nl + 2) * (nl + 2));
  }
  for (int Ml = Mblocks * 2;; Ml /= 2) {
    p.gm.push_back(Ml);
    p.cells.push_back((long)Ml * Ml * Ml);
    if (Ml == 1 || Ml % 2 == 1) break;
  }
  return p;
}

template <typename T>
BlockCycle<T> make_cycle(const DevMesh& m, const std::vector<void*>& bufs, const Plan& P, double h, cudaStream_t s) {
  BlockCycle<T> C;
  C.m = m;
  C.B = m.B;
  C.s = s;
  C.tail.s = s;
  size_t k = 0;
  for (size_t l = 0; l < P.bn.size(); ++l, ++k)
    C.blk.push_back(BLevel<T>{P.bn[l], h * (double)(1L << l), static_cast<T*>(bufs[3 * k]),
                              static_cast<T*>(bufs[3 * k + 1]), static_cast<T*>(bufs[3 * k + 2])});
  for (size_t l = 0; l < P.gm.size(); ++l, ++k)
    C.tail.lv.push_back(Level<T>{P.gm[l], h * (double)(1L << k), static_cast<T*>(bufs[3 * k]),
                                 static_cast<T*>(bufs[3 * k + 1]), static_cast<T*>(bufs[3 * k + 2])});
  return C;
}

// mean of a compact array (count doubles) into *out
void mean_of(const double* a, long count, double* red, double* out, cudaStream_t s) {
  reduce_kernel<<<1024, kRedThreads, 0, s>>>(a, nullptr, count, 0, 0.0, 0, red);
  fold_kernel<<<1, kRedThreads, 0, s>>>(red, 1024, 0, 1.0 / (double)count, out);
}

}  // namespace

cudaError_t poisson_solve(PoissonScratch** scratch, const DevMesh& m, int M, double h, const double* f_leaves,
                          double* phi_leaves, int cycles, int inner, double* resid_host, cudaStream_t s) {
  const int n = m.n, B = m.B;
  const Plan P = plan_levels(B, n, M / n);
  if (!*scratch) *scratch = new PoissonScratch();
  PoissonScratch* S = *scratch;
  // float64 level 0 always; the float64 hierarchy for float64 cycles, the
  // float32 hierarchy for mixed precision
  cudaError_t e = alloc_levels(S->d64, inner == 8 ? P.cells : std::vector<long>{P.cells[0]}, sizeof(double));
  if (e == cudaSuccess && inner == 4) e = alloc_levels(S->d32, P.cells, sizeof(float));
  if (e == cudaSuccess && !S->red) e = cudaMalloc(&S->red, sizeof(double) * (1024 + 2));
  if (e != cudaSuccess) return e;
  double* scalar = S->red + 1024;
  const long nl = (long)B * n * n * n;
  const long p0 = P.cells[0];
  const double ih2 = 1.0 / (h * h);
  BlockCycle<double> C64;
  BlockCycle<float> C32;
  // level 0 in float64: f without its mean, phi = 0
  BLevel<double> L0{n, h, static_cast<double*>(S->d64[0]), static_cast<double*>(S->d64[1]),
                    static_cast<double*>(S->d64[2])};
  if (inner == 8) {
    C64 = make_cycle<double>(m, S->d64, P, h, s);
    L0 = C64.blk[0];
  } else {
    C32 = make_cycle<float>(m, S->d32, P, h, s);
    C64.m = m;
    C64.B = B;
    C64.s = s;
  }
  mean_of(f_leaves, nl, S->red, scalar, s);
  blk_from_leaves_kernel<<<blocks_for(nl), 256, 0, s>>>(f_leaves, L0.f, n, B, scalar);
  fill_kernel<double><<<blocks_for(p0), 256, 0, s>>>(L0.phi, p0, 0.0);
  for (int k = 0; k < cycles; ++k) {
    if (inner == 8) {
      C64.blk[0].phi = L0.phi;
      C64.blk[0].tmp = L0.tmp;
      C64.vcycle(0);
      L0.phi = C64.blk[0].phi;
      L0.tmp = C64.blk[0].tmp;
    } else {
      BLevel<float>& F = C32.blk[0];
      C64.refresh(L0, L0.phi);
      blk_residual_f32_kernel<<<blocks_for(nl), 256, 0, s>>>(L0.phi, L0.f, F.f, n, B, ih2);
      fill_kernel<float><<<blocks_for(p0), 256, 0, s>>>(F.phi, p0, 0.0f);
      C32.vcycle(0);
      blk_correct_kernel<<<blocks_for(nl), 256, 0, s>>>(L0.phi, F.phi, n, B);
    }
    if (resid_host) {
      C64.refresh(L0, L0.phi);
      blk_resmax_kernel<<<1024, kRedThreads, 0, s>>>(L0.phi, L0.f, n, B, ih2, S->red);
      fold_kernel<<<1, kRedThreads, 0, s>>>(S->red, 1024, 1, 1.0, scalar + 1);
      e = cudaMemcpyAsync(resid_host + k, scalar + 1, sizeof(double), cudaMemcpyDeviceToHost, s);
      if (e != cudaSuccess) return e;
    }
  }
  blk_to_leaves_kernel<<<blocks_for(nl), 256, 0, s>>>(L0.phi, phi_leaves, n, B);
  mean_of(phi_leaves, nl, S->red, scalar, s);
  add_kernel<<<blocks_for(nl), 256, 0, s>>>(phi_leaves, nl, scalar, 1.0);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (resid_host) e = cudaStreamSynchronize(s);
  return e;
}

}  // namespace cello
