// Float64 sweep and the precision-generic kernels (refresh, reductions,
// flags, flux correction).  Built without FMA contraction so that float64
// results round exactly like the same formulas evaluated term by term.
#define CELLO_DEFINE_FINISH_KERNEL
#include "kernels.cuh"
#include "adjoint_kernels.cuh"

namespace cello {

// Float64 sweep variants: {pencils per CTA, min resident CTAs per SM, persistent}.
static const SweepVariant kVariants64[] = {{8, 2, false}, {8, 2, true}};
constexpr int kNV64 = 2;
static int g_resident64[3];

static int nb_index64(int n) { return n == 8 ? 0 : (n == 16 ? 1 : 2); }

template <int NB, int RS>
static constexpr size_t sweep_smem64() {
  constexpr int N = NB + 2 * kGhosts;
  return sizeof(double) * sweep_arrays(RS) * N * 8;
}

template <int NB, int RS>
static void set_smem_attr64() {
  cudaFuncSetAttribute(sweep_kernel<double, NB, 8, 2, RS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sweep_smem64<NB, RS>());
}

template <int NB>
static void prepare_nb64(int sms) {
  constexpr int N = NB + 2 * kGhosts;
  set_smem_attr64<NB, 0>();
  set_smem_attr64<NB, 1>();
  set_smem_attr64<NB, 2>();
  set_smem_attr64<NB, 3>();
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel<double, NB, 8, 2, 0>, N * 8, sweep_smem64<NB, 0>());
  g_resident64[nb_index64(NB)] = (nb > 0 ? nb : 1) * sms;
}

template <int NB>
static void launch_nb64(const DevMesh& m, SweepParams p, int pencils, cudaStream_t s) {
  constexpr int N = NB + 2 * kGhosts;
  const int v = (p.variant >= 0 && p.variant < kNV64) ? p.variant : 0;
  p.tiles_per_leaf = (pencils + 7) / 8;
  p.n_items = p.nleaf * p.tiles_per_leaf;
  if (p.n_items <= 0) return;
  p.div_tiles = FastDiv::make((unsigned)p.tiles_per_leaf);
  p.div_cb = FastDiv::make((unsigned)(p.b1 - p.b0));
  int grid = p.n_items;
  if (kVariants64[v].persistent && p.work) {
    cudaMemsetAsync(p.work, 0, sizeof(unsigned), s);
    grid = g_resident64[nb_index64(NB)] < grid ? g_resident64[nb_index64(NB)] : grid;
  } else {
    p.work = nullptr;
  }
  switch (method_code(m.riemann, m.steepen, m.nf == 6)) {
    case 0: sweep_kernel<double, NB, 8, 2, 0><<<grid, N * 8, sweep_smem64<NB, 0>(), s>>>(m, p); break;
    case 1: sweep_kernel<double, NB, 8, 2, 1><<<grid, N * 8, sweep_smem64<NB, 1>(), s>>>(m, p); break;
    case 2: sweep_kernel<double, NB, 8, 2, 2><<<grid, N * 8, sweep_smem64<NB, 2>(), s>>>(m, p); break;
    case 3: sweep_kernel<double, NB, 8, 2, 3><<<grid, N * 8, sweep_smem64<NB, 3>(), s>>>(m, p); break;
    default: launch_sweep_de_f64<NB>(m, p, grid, s); break;   // dual energy (k_de_f64.cu)
  }
}

int sweep_variant_count_f64() { return kNV64; }
SweepVariant sweep_variant_f64(int v) { return kVariants64[v]; }

void launch_sweep_f64(const DevMesh& m, const SweepParams& p, int pencils, cudaStream_t s) {
  switch (m.n) {
    case 8: launch_nb64<8>(m, p, pencils, s); break;
    case 16: launch_nb64<16>(m, p, pencils, s); break;
    case 32: launch_nb64<32>(m, p, pencils, s); break;
  }
}

template <int NB, int P>
static size_t adj_smem() {
  constexpr int N = NB + 2 * kGhosts;
  return sizeof(double) * (10 * N * (P + 1) + (NB + 1) * 40 * P);
}

template <int NB>
static void prepare_adj() {
  cudaFuncSetAttribute(adjoint_sweep_kernel<double, NB, kAdjPencils>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)adj_smem<NB, kAdjPencils>());
}

template <int NB>
static void adj_sweep_n(const DevMesh& m, const AdjSweepParams& p, cudaStream_t s) {
  constexpr int N = NB + 2 * kGhosts;
  adjoint_sweep_kernel<double, NB, kAdjPencils><<<p.n_items, N * kAdjPencils, adj_smem<NB, kAdjPencils>(), s>>>(m, p);
}

void launch_adjoint_sweep_f64(const DevMesh& m, const AdjSweepParams& p, cudaStream_t s) {
  if (p.n_items <= 0) return;
  switch (m.n) {
    case 8: adj_sweep_n<8>(m, p, s); break;
    case 16: adj_sweep_n<16>(m, p, s); break;
    case 32: adj_sweep_n<32>(m, p, s); break;
  }
}


void prepare_kernels_f64() {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  prepare_nb64<8>(sms);
  prepare_nb64<16>(sms);
  prepare_nb64<32>(sms);
  prepare_adj<8>();
  prepare_adj<16>();
  prepare_adj<32>();
}

template <typename T, int NB, int NF>
static void refresh_nf(const DevMesh& m, T* U, int leaf0, int nleaf, const int* slow, int nslow, int phases,
                       cudaStream_t s) {
  constexpr int G = kGhosts, N = NB + 2 * G;
  auto blocks = [](long threads, int per) { return (unsigned)((threads + per - 1) / per); };
  if ((phases & kRefreshSlow) && nslow > 0) refresh_slow_kernel<T, NB, NF><<<nslow, 128, 0, s>>>(m, U, slow, nslow);
  if (nleaf <= 0) return;
  if (phases & kRefreshX)   // float32: one thread per row pair (see refresh_x_kernel)
    refresh_x_kernel<T, NB, NF><<<blocks((long)nleaf * NB * (sizeof(T) == 4 ? NB / 2 : NB), 256), 256, 0, s>>>(
        m, U, leaf0, nleaf);
  constexpr int S = Sector<T>::kCells;
  if (phases & kRefreshY)
    refresh_y_kernel<T, NB, NF><<<blocks((long)nleaf * 2 * NF * NB * (G * N / S), 256), 256, 0, s>>>(m, U, leaf0,
                                                                                                   nleaf);
  if (phases & kRefreshZ)
    refresh_z_kernel<T, NB, NF><<<blocks((long)nleaf * 2 * NF * (G * N * N / S), 256), 256, 0, s>>>(m, U, leaf0,
                                                                                                    nleaf);
}

template <typename T, int NB>
static void refresh_n(const DevMesh& m, T* U, int leaf0, int nleaf, const int* slow, int nslow, int phases,
                      cudaStream_t s) {
  if (m.nf == 6) refresh_nf<T, NB, 6>(m, U, leaf0, nleaf, slow, nslow, phases, s);
  else refresh_nf<T, NB, 5>(m, U, leaf0, nleaf, slow, nslow, phases, s);
}

template <typename T>
static void refresh_t(const DevMesh& m, T* U, int leaf0, int nleaf, const int* slow, int nslow, int phases,
                      cudaStream_t s) {
  switch (m.n) {
    case 8: refresh_n<T, 8>(m, U, leaf0, nleaf, slow, nslow, phases, s); break;
    case 16: refresh_n<T, 16>(m, U, leaf0, nleaf, slow, nslow, phases, s); break;
    case 32: refresh_n<T, 32>(m, U, leaf0, nleaf, slow, nslow, phases, s); break;
  }
}

void launch_refresh_f32(const DevMesh& m, float* U, int leaf0, int nleaf, const int* slow, int nslow,
                        int phases, cudaStream_t s) {
  refresh_t<float>(m, U, leaf0, nleaf, slow, nslow, phases, s);
}
void launch_refresh_f64(const DevMesh& m, double* U, int leaf0, int nleaf, const int* slow, int nslow,
                        int phases, cudaStream_t s) {
  refresh_t<double>(m, U, leaf0, nleaf, slow, nslow, phases, s);
}


template <typename T, int NB>
static void reduce_n(const DevMesh& m, const void* U, double* partials, int leaf0, int nleaf, int g,
                     cudaStream_t s) {
  if (m.nf == 6)
    reduce_partials_kernel<T, NB, 6><<<g, kReduceThreads, 0, s>>>(m, static_cast<const T*>(U), partials, leaf0, nleaf);
  else
    reduce_partials_kernel<T, NB><<<g, kReduceThreads, 0, s>>>(m, static_cast<const T*>(U), partials, leaf0, nleaf);
}

void launch_reduce_range(const DevMesh& m, const void* U, int precision, double cfl, double* partials, int leaf0,
                         int nleaf, double* dt_next, double* totals, cudaStream_t s, int grid) {
  if (nleaf <= 0) return;
  const int g = (grid > 0 && grid < nleaf) ? grid : nleaf;
#define CELLO_RED(T)                                                          \
  switch (m.n) {                                                              \
    case 8: reduce_n<T, 8>(m, U, partials, leaf0, nleaf, g, s); break;        \
    case 16: reduce_n<T, 16>(m, U, partials, leaf0, nleaf, g, s); break;      \
    case 32: reduce_n<T, 32>(m, U, partials, leaf0, nleaf, g, s); break;      \
  }
  if (precision == 4) {
    launch_reduce_partials_f32(m, static_cast<const float*>(U), partials, leaf0, nleaf, g, s);
  } else {
    CELLO_RED(double)
  }
#undef CELLO_RED
  reduce_finish_kernel<<<1, 1024, 0, s>>>(partials + (long)leaf0 * 6, nleaf, cfl, dt_next, totals);
}

void launch_reduce(const DevMesh& m, const void* U, int precision, double cfl, double* partials,
                   double* dt_next, double* totals, cudaStream_t s, int grid) {
  launch_reduce_range(m, U, precision, cfl, partials, 0, m.B, dt_next, totals, s, grid);
}

template <typename T, int NB>
static void adj_refresh_n(const DevMesh& m, T* lam, cudaStream_t s) {
  const long cells = (long)m.B * NB * NB * NB;
  adjoint_refresh_gather_kernel<T, NB><<<(unsigned)((cells + 255) / 256), 256, 0, s>>>(m, lam);
  constexpr int N = NB + 2 * kGhosts;
  const long ng = (long)m.B * ((long)N * N * N - (long)NB * NB * NB);
  zero_ghosts_kernel<T, NB><<<(unsigned)((ng + 255) / 256), 256, 0, s>>>(lam, m.B);
}

template <typename T, int NB>
static void zero_n(const DevMesh& m, T* lam, cudaStream_t s) {
  constexpr int N = NB + 2 * kGhosts;
  const long ng = (long)m.B * ((long)N * N * N - (long)NB * NB * NB);
  zero_ghosts_kernel<T, NB><<<(unsigned)((ng + 255) / 256), 256, 0, s>>>(lam, m.B);
}

void launch_adjoint_refresh(const DevMesh& m, void* lam, int precision, cudaStream_t s) {
  if (m.B <= 0) return;
#define CELLO_AR(T)                                                  \
  switch (m.n) {                                                     \
    case 8: adj_refresh_n<T, 8>(m, static_cast<T*>(lam), s); break;  \
    case 16: adj_refresh_n<T, 16>(m, static_cast<T*>(lam), s); break;\
    case 32: adj_refresh_n<T, 32>(m, static_cast<T*>(lam), s); break;\
  }
  if (precision == 4) { CELLO_AR(float) } else { CELLO_AR(double) }
#undef CELLO_AR
}

template <typename T, int NB>
static void adj_scatter_n(const DevMesh& m, const T* U, T* lam, cudaStream_t s) {
  constexpr int N = NB + 2 * kGhosts;
  const long ng = (long)m.B * ((long)N * N * N - (long)NB * NB * NB);
  adjoint_refresh_scatter_kernel<T, NB><<<(unsigned)((ng + 255) / 256), 256, 0, s>>>(m, U, lam);
  zero_ghosts_kernel<T, NB><<<(unsigned)((ng + 255) / 256), 256, 0, s>>>(lam, m.B);
}

void launch_adjoint_refresh_scatter(const DevMesh& m, const void* U, void* lam, int precision, cudaStream_t s) {
  if (m.B <= 0) return;
#define CELLO_AS(T)                                                                                        \
  switch (m.n) {                                                                                           \
    case 8: adj_scatter_n<T, 8>(m, static_cast<const T*>(U), static_cast<T*>(lam), s); break;             \
    case 16: adj_scatter_n<T, 16>(m, static_cast<const T*>(U), static_cast<T*>(lam), s); break;           \
    case 32: adj_scatter_n<T, 32>(m, static_cast<const T*>(U), static_cast<T*>(lam), s); break;           \
  }
  if (precision == 4) { CELLO_AS(float) } else { CELLO_AS(double) }
#undef CELLO_AS
}

void launch_fluxcorr_adjoint(const DevMesh& m, const void* lam, int precision, const CoarseFace* faces, int nfaces,
                             double* regb, const double* dt, cudaStream_t s) {
  if (nfaces <= 0) return;
  const long threads = (long)nfaces * m.n * m.n;
  const unsigned grid = (unsigned)((threads + 255) / 256);
#define CELLO_FA(T, NB) \
  fluxcorr_adjoint_kernel<T, NB><<<grid, 256, 0, s>>>(m, static_cast<const T*>(lam), faces, nfaces, regb, dt)
#define CELLO_FA_T(T)                       \
  switch (m.n) {                            \
    case 8: CELLO_FA(T, 8); break;          \
    case 16: CELLO_FA(T, 16); break;        \
    case 32: CELLO_FA(T, 32); break;        \
  }
  if (precision == 4) { CELLO_FA_T(float) } else { CELLO_FA_T(double) }
#undef CELLO_FA_T
#undef CELLO_FA
}

void launch_zero_ghosts(const DevMesh& m, void* lam, int precision, cudaStream_t s) {
  if (m.B <= 0) return;
#define CELLO_ZG(T)                                           \
  switch (m.n) {                                              \
    case 8: zero_n<T, 8>(m, static_cast<T*>(lam), s); break;  \
    case 16: zero_n<T, 16>(m, static_cast<T*>(lam), s); break;\
    case 32: zero_n<T, 32>(m, static_cast<T*>(lam), s); break;\
  }
  if (precision == 4) { CELLO_ZG(float) } else { CELLO_ZG(double) }
#undef CELLO_ZG
}

void launch_remap(const DevMesh& neu, const DevMesh& old, const void* Uold, void* Unew, const RemapEntry* map,
                  int precision, cudaStream_t s) {
  const long threads = (long)neu.B * neu.n * neu.n * neu.n;
  if (threads <= 0) return;
  const unsigned grid = (unsigned)((threads + 255) / 256);
#define CELLO_RM(T, NB)                                                                                      \
  if (neu.nf == 6)                                                                                          \
    remap_kernel<T, NB, 6><<<grid, 256, 0, s>>>(neu, old, static_cast<const T*>(Uold), static_cast<T*>(Unew), map); \
  else                                                                                                      \
    remap_kernel<T, NB><<<grid, 256, 0, s>>>(neu, old, static_cast<const T*>(Uold), static_cast<T*>(Unew), map)
#define CELLO_RM_T(T)                       \
  switch (neu.n) {                          \
    case 8: CELLO_RM(T, 8); break;          \
    case 16: CELLO_RM(T, 16); break;        \
    case 32: CELLO_RM(T, 32); break;        \
  }
  if (precision == 4) { CELLO_RM_T(float) } else { CELLO_RM_T(double) }
#undef CELLO_RM_T
#undef CELLO_RM
}

void launch_flags(const DevMesh& m, const void* U, int precision, int field, double tau, double tau_c,
                  int8_t* flags, cudaStream_t s) {
  if (m.B <= 0) return;
  const double thr = 2.0 * tau, thr_c = 2.0 * tau_c;
#define CELLO_FLG(T, NB)                                                                                     \
  if (m.nf == 6)                                                                                            \
    flags_kernel<T, NB, 6><<<m.B, 256, 0, s>>>(m, static_cast<const T*>(U), field, thr, thr_c, flags);     \
  else                                                                                                      \
    flags_kernel<T, NB><<<m.B, 256, 0, s>>>(m, static_cast<const T*>(U), field, thr, thr_c, flags)
#define CELLO_FLG_T(T)                        \
  switch (m.n) {                              \
    case 8: CELLO_FLG(T, 8); break;           \
    case 16: CELLO_FLG(T, 16); break;         \
    case 32: CELLO_FLG(T, 32); break;         \
  }
  if (precision == 4) { CELLO_FLG_T(float) } else { CELLO_FLG_T(double) }
#undef CELLO_FLG_T
#undef CELLO_FLG
}

void launch_fluxcorr(const DevMesh& m, void* U, int precision, const CoarseFace* faces, const int* group_start,
                     int ngroups, const double* reg, const double* dt, cudaStream_t s) {
  if (ngroups <= 0) return;
#define CELLO_FC(T, NB)                                                                                      \
  if (m.nf == 6)                                                                                            \
    fluxcorr_kernel<T, NB, 6><<<ngroups, 256, 0, s>>>(m, static_cast<T*>(U), faces, group_start, reg, dt);  \
  else                                                                                                      \
    fluxcorr_kernel<T, NB><<<ngroups, 256, 0, s>>>(m, static_cast<T*>(U), faces, group_start, reg, dt)
#define CELLO_FC_T(T)                       \
  switch (m.n) {                            \
    case 8: CELLO_FC(T, 8); break;          \
    case 16: CELLO_FC(T, 16); break;        \
    case 32: CELLO_FC(T, 32); break;        \
  }
  if (precision == 4) { CELLO_FC_T(float) } else { CELLO_FC_T(double) }
#undef CELLO_FC_T
#undef CELLO_FC
}

}  // namespace cello

// ---------------------------------------------------------------------------
// Sharded step: leaf interiors and flux registers to and from flat buffers.
namespace cello {
namespace {

// Leaf interiors <-> buf[count][nf][n^3] (x fastest), four cells per thread
// (16-byte vectors: interior rows start at x = G, a multiple of four).
template <typename T, int NB>
__global__ void __launch_bounds__(256) halo_copy_kernel(T* U, const int* ids, long count, int nf, T* buf, int pack) {
  constexpr int G = kGhosts, N = NB + 2 * G, Q = NB / 4;
  constexpr long SLAB = (long)N * N * N;
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= count * nf * NB * NB * Q) return;
  const int q = (int)(gid % Q);
  const int row = (int)((gid / Q) % (NB * NB));
  const long kf = gid / ((long)Q * NB * NB);
  const int f = (int)(kf % nf);
  const long k = kf / nf;
  T* u = U + ((long)ids[k] * nf + f) * SLAB + ((long)(row / NB + G) * N + (row % NB + G)) * N + G + 4 * q;
  T* b = buf + (kf * NB * NB + row) * NB + 4 * q;
  Vec4<T> v;
  if (pack) {
    v.load(u);
    v.store(b);
  } else {
    v.load(b);
    v.store(u);
  }
}

__global__ void __launch_bounds__(256) flux_copy_kernel(double* reg, const int* slots, long count, long per,
                                                        double* buf, int pack) {
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= count * per) return;
  double* r = reg + (long)slots[gid / per] * per + gid % per;
  if (pack) buf[gid] = *r;
  else *r = buf[gid];
}

template <typename T>
void halo_copy_t(const DevMesh& m, T* U, const int* ids, long count, T* buf, int pack, cudaStream_t s) {
  const long threads = count * m.nf * (long)m.n * m.n * (m.n / 4);
  const unsigned grid = (unsigned)((threads + 255) / 256);
  switch (m.n) {
    case 8: halo_copy_kernel<T, 8><<<grid, 256, 0, s>>>(U, ids, count, m.nf, buf, pack); break;
    case 16: halo_copy_kernel<T, 16><<<grid, 256, 0, s>>>(U, ids, count, m.nf, buf, pack); break;
    case 32: halo_copy_kernel<T, 32><<<grid, 256, 0, s>>>(U, ids, count, m.nf, buf, pack); break;
  }
}

}  // namespace

void launch_halo_copy(const DevMesh& m, void* U, int precision, const int* ids, long count, void* buf, int pack,
                      cudaStream_t s) {
  if (count <= 0) return;
  if (precision == 4) halo_copy_t<float>(m, static_cast<float*>(U), ids, count, static_cast<float*>(buf), pack, s);
  else halo_copy_t<double>(m, static_cast<double*>(U), ids, count, static_cast<double*>(buf), pack, s);
}

// The interior cells of every (leaf, field) slab from src to dst, one
// 16-byte chunk of an interior row per thread (NB cells: 8 chunks in float32,
// 16 in float64; every chunk starts 16-byte aligned since rows are N cells
// and the interior starts G = 4 cells in).  With one side the mapped address
// of a page-locked host buffer, the SMs move the interior across the host
// link as coalesced 128-byte requests and no ghost cell crosses it.
template <typename T, int NB>
__global__ void __launch_bounds__(256) interior_copy_kernel(const T* __restrict__ src, T* __restrict__ dst,
                                                            long slabs) {
  constexpr int G = kGhosts, N = NB + 2 * G, V = 16 / (int)sizeof(T), C = NB / V;
  constexpr long SLAB = (long)N * N * N;
  const long gid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= slabs * NB * NB * C) return;
  const int c = (int)(gid % C);
  long q = gid / C;
  const int y = G + (int)(q % NB);
  q /= NB;
  const int z = G + (int)(q % NB);
  const long slab = q / NB;
  const long o = slab * SLAB + ((long)z * N + y) * N + G + (long)c * V;
  *reinterpret_cast<float4*>(dst + o) = *reinterpret_cast<const float4*>(src + o);
}

template <typename T>
static void interior_copy_t(int n, const T* src, T* dst, long slabs, cudaStream_t s) {
  const long threads = slabs * n * n * (n * (long)sizeof(T) / 16);
  const unsigned grid = (unsigned)((threads + 255) / 256);
  switch (n) {
    case 8: interior_copy_kernel<T, 8><<<grid, 256, 0, s>>>(src, dst, slabs); break;
    case 16: interior_copy_kernel<T, 16><<<grid, 256, 0, s>>>(src, dst, slabs); break;
    case 32: interior_copy_kernel<T, 32><<<grid, 256, 0, s>>>(src, dst, slabs); break;
  }
}

void launch_interior_copy(const DevMesh& m, const void* src, void* dst, int precision, cudaStream_t s) {
  const long slabs = (long)m.B * m.nf;
  if (slabs <= 0) return;
  if (precision == 4) interior_copy_t<float>(m.n, static_cast<const float*>(src), static_cast<float*>(dst), slabs, s);
  else interior_copy_t<double>(m.n, static_cast<const double*>(src), static_cast<double*>(dst), slabs, s);
}

void launch_flux_copy(double* reg, const int* slots, long count, long per, double* buf, int pack, cudaStream_t s) {
  if (count <= 0) return;
  flux_copy_kernel<<<(unsigned)((count * per + 255) / 256), 256, 0, s>>>(reg, slots, count, per, buf, pack);
}

}  // namespace cello
