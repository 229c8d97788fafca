// Tracer particles (Sec. II.B: Lagrangian particles that move between
// Blocks; Sec. III: the hydro scaling workload carries tracers).  Positions
// are float64 in structure-of-arrays form pos[3][count]; each tracer keeps
// the index of the leaf that contains it, -1 once lost through an outflow
// face.  Built without FMA contraction: every position is the same float64
// arithmetic as a term-by-term evaluation.
//
// Lookup: the block index at max_level of the point, b = floor((x - lo) /
// w) clamped into the root array, gives a Morton key; the containing leaf is
// the last leaf whose key does not exceed it (leaves tile the domain and
// are sorted by key).  Velocity: momentum over floored density, trilinear
// between the cell centres of the leaf's padded block (ghosts refreshed),
// along x, then y, then z.  Push: x += dt u, periodic wrap or outflow loss,
// lookup again (migration).
//
// Where the block width at max_level and the level-0 cell width are powers
// of two (a box whose extent over the root count is one), each division by a
// width is a multiplication by its reciprocal, also a power of two: both
// give the correctly rounded value of the same exact quotient, so the
// results are bit-identical, and six float64 divisions per tracer leave the
// slow float64 pipe.
#include "cello_internal.h"
#include "morton.h"
#include "ppm.cuh"

namespace cello {
namespace {

struct PartMesh {
  DevMesh m;
  const unsigned long long* keys;
  double lo[3], hi[3];
  double w;   // block width at max_level
  double inv_w, inv_dx0;   // 1 / w and 1 / (level-0 cell width), exact when pow2
  bool pow2;               // both widths powers of two
};

__device__ __forceinline__ double over_w(const PartMesh& P, double d) { return P.pow2 ? d * P.inv_w : d / P.w; }

__device__ __forceinline__ int locate_point(const PartMesh& P, const double x[3]) {
  unsigned b[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const long nb = (long)P.m.root[a] << P.m.max_level;
    long v = (long)floor(over_w(P, x[a] - P.lo[a]));
    v = v < 0 ? 0 : (v > nb - 1 ? nb - 1 : v);
    b[a] = (unsigned)v;
  }
  const unsigned long long k = morton3(b[0], b[1], b[2]);
  int lo = 0, hi = P.m.B;   // first key > k
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (P.keys[mid] <= k) lo = mid + 1;
    else hi = mid;
  }
  return lo - 1;
}

// 1/rho: the correctly rounded float32 reciprocal of float32(rho) refined by
// two float64 Newton steps (within 2 ulp), a handful of float64 operations
// where a float64 division costs many on this part's slow float64 pipe.
__device__ __forceinline__ double reciprocal(double rho) {
  double r = (double)__frcp_rn((float)rho);
  r = r * (2.0 - rho * r);
  return r * (2.0 - rho * r);
}

// Velocity (3 components) of the cell at offset o of a padded block.
template <typename T>
__device__ __forceinline__ void cell_velocity(const T* blk, long SLAB, long o, double v[3]) {
  const double r = (double)blk[o];
  const double ir = reciprocal(r > kRhoFloor ? r : kRhoFloor);
#pragma unroll
  for (int c = 0; c < 3; ++c) v[c] = (double)blk[(1 + c) * SLAB + o] * ir;
}

// Three CTAs of 256 per SM (80 registers, a few spilled to L1): the corner
// gathers of randomly placed tracers are latency bound, and the extra warps
// hide more of it.
template <typename T>
__global__ void __launch_bounds__(256, 3) particles_push_kernel(PartMesh P, const T* U, double* pos, int* leaf, long count,
                                      const double* dt_dev) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int b = leaf[i];
  if (b < 0 || b >= P.m.B) return;
  const DevMesh& m = P.m;
  const int n = m.n, g = m.g, N = m.N;
  const long SLAB = (long)N * N * N;
  const int4 lf = m.leaf[b];
  const double dx = ldexp(m.dx0, -lf.x);
  const double inv_dx = ldexp(P.inv_dx0, lf.x);
  const int lidx[3] = {lf.y, lf.z, lf.w};
  double x[3], f[3];
  int i0[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    x[a] = pos[a * count + i];
    const double d = x[a] - (P.lo[a] + (double)(lidx[a] * n) * dx);
    const double s = (P.pow2 ? d * inv_dx : d / dx) - 0.5;
    const double c = floor(s);
    i0[a] = (int)c + g;
    f[a] = s - c;
  }
  const T* blk = U + (long)b * m.nf * SLAB;
  const long o000 = ((long)i0[2] * N + i0[1]) * N + i0[0];
  const long sx = 1, sy = N, sz = (long)N * N;
  const double dt = *dt_dev;
  // the eight corner velocities, x fastest: corner (dz, dy, dx) at index 4 dz + 2 dy + dx
  double cv[8][3];
#pragma unroll
  for (int q = 0; q < 8; ++q) cell_velocity(blk, SLAB, o000 + (q >> 2) * sz + ((q >> 1) & 1) * sy + (q & 1) * sx, cv[q]);
  bool lost = false;
#pragma unroll
  for (int comp = 0; comp < 3; ++comp) {
    const double fx = f[0], fy = f[1], fz = f[2];
    const double c00 = cv[0][comp] * (1.0 - fx) + cv[1][comp] * fx;
    const double c10 = cv[2][comp] * (1.0 - fx) + cv[3][comp] * fx;
    const double c01 = cv[4][comp] * (1.0 - fx) + cv[5][comp] * fx;
    const double c11 = cv[6][comp] * (1.0 - fx) + cv[7][comp] * fx;
    const double c0 = c00 * (1.0 - fy) + c10 * fy;
    const double c1 = c01 * (1.0 - fy) + c11 * fy;
    const double v = c0 * (1.0 - fz) + c1 * fz;
    double xn = x[comp] + dt * v;
    const double ext = P.hi[comp] - P.lo[comp];
    if (m.bc[comp] == CELLO_PERIODIC) {
      xn = xn < P.lo[comp] ? xn + ext : (xn >= P.hi[comp] ? xn - ext : xn);
    } else if (xn < P.lo[comp] || xn >= P.hi[comp]) {
      lost = true;
    }
    x[comp] = xn;
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) pos[a * count + i] = x[a];
  leaf[i] = lost ? -1 : locate_point(P, x);
}

__global__ void particles_locate_kernel(PartMesh P, const double* pos, int* leaf, long count) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const double x[3] = {pos[i], pos[count + i], pos[2 * count + i]};
  leaf[i] = locate_point(P, x);
}

bool is_pow2(double v) {
  int e;
  return v > 0.0 && std::frexp(v, &e) == 0.5;
}

PartMesh part_mesh(const DevMesh& m, const unsigned long long* keys, const double lo[3], const double hi[3]) {
  PartMesh P{m, keys, {lo[0], lo[1], lo[2]}, {hi[0], hi[1], hi[2]}, ldexp((hi[0] - lo[0]) / m.root[0], -m.max_level)};
  P.pow2 = is_pow2(P.w) && is_pow2(m.dx0);
  P.inv_w = 1.0 / P.w;
  P.inv_dx0 = 1.0 / m.dx0;
  return P;
}

}  // namespace

void launch_particles_locate(const DevMesh& m, const unsigned long long* keys, const double lo[3], const double hi[3],
                             const double* pos, int* leaf, long count, cudaStream_t s) {
  if (count <= 0) return;
  const PartMesh P = part_mesh(m, keys, lo, hi);
  particles_locate_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(P, pos, leaf, count);
}

void launch_particles_push(const DevMesh& m, const unsigned long long* keys, const double lo[3], const double hi[3],
                           const void* U, int precision, double* pos, int* leaf, long count, const double* dt,
                           cudaStream_t s) {
  if (count <= 0) return;
  const PartMesh P = part_mesh(m, keys, lo, hi);
  const unsigned grid = (unsigned)((count + 255) / 256);
  if (precision == 4)
    particles_push_kernel<float><<<grid, 256, 0, s>>>(P, static_cast<const float*>(U), pos, leaf, count, dt);
  else
    particles_push_kernel<double><<<grid, 256, 0, s>>>(P, static_cast<const double*>(U), pos, leaf, count, dt);
}

}  // namespace cello
