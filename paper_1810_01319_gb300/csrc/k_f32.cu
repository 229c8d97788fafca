// Float32 PPM sweep (bulk arithmetic in float32, FMA contraction allowed).
#include "kernels.cuh"
#include "adjoint_kernels.cuh"

namespace cello {

// Float32 sweep variants.  Shared-memory form: {pencils per CTA, min
// resident CTAs per SM}; register-streaming form: {CTA size = pencils per
// CTA, min resident CTAs per SM}; each without and with the persistent
// work-counter schedule.
static const SweepVariant kVariants[] = {
    {8, 3, false, false},  {8, 4, false, false},  {4, 6, false, false}, {16, 1, false, false},
    {4, 8, false, false},  {16, 2, false, false}, {64, 8, false, true}, {128, 4, false, true},
    {64, 6, false, true},  {32, 16, false, true}, {64, 8, false, true, 3}, {64, 6, false, true, 3},
    {8, 3, true, false},   {8, 4, true, false},   {4, 6, true, false},  {16, 1, true, false},
    {4, 8, true, false},   {16, 2, true, false},  {64, 8, true, true},  {128, 4, true, true},
    {64, 6, true, true},   {32, 16, true, true},  {64, 8, true, true, 3},  {64, 6, true, true, 3},
};
constexpr int kNT = 12;  // distinct kernel instantiations; variant v uses template v % kNT
constexpr int kNV = sizeof(kVariants) / sizeof(kVariants[0]);
static int g_resident[3][kNV];   // resident CTAs per GPU by [n index][variant], from the occupancy API

static int nb_index(int n) { return n == 8 ? 0 : (n == 16 ? 1 : 2); }

// Shared memory of the shared-memory form: sweep_arrays(RS) arrays of N x P
// values (21; 24 with contact steepening).
template <int NB, int P, int RS>
static constexpr size_t sweep_smem() {
  constexpr int N = NB + 2 * kGhosts;
  return sizeof(float) * sweep_arrays(RS) * N * P;
}

template <int NB, int P, int MINB, int RS>
static void set_smem_attr() {
  cudaFuncSetAttribute(sweep_kernel<float, NB, P, MINB, RS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sweep_smem<NB, P, RS>());
}

template <int NB, int P, int MINB>
static void prepare_variant(int v, int sms) {
  constexpr int N = NB + 2 * kGhosts;
  set_smem_attr<NB, P, MINB, 0>();
  set_smem_attr<NB, P, MINB, 1>();
  set_smem_attr<NB, P, MINB, 2>();
  set_smem_attr<NB, P, MINB, 3>();
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel<float, NB, P, MINB, 0>, N * P,
                                                sweep_smem<NB, P, 0>());
  g_resident[nb_index(NB)][v] = (nb > 0 ? nb : 1) * sms;
}

// Dynamic shared memory of the streaming form: the staged form keeps three
// groups of four cells of five fields per thread, and the updated group.
template <int CT, int VEC>
static constexpr size_t stream_smem() {
  return VEC == 3 ? sizeof(float4) * 4 * 5 * CT : 0;
}

template <int NB, int CT, int MINB, int VEC>
static void prepare_stream_variant(int v, int sms) {
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_stream_kernel<float, NB, CT, MINB, VEC, 0>, CT,
                                                stream_smem<CT, VEC>());
  g_resident[nb_index(NB)][v] = (nb > 0 ? nb : 1) * sms;
}

// Work items, grid and schedule of one launch; false if there is no work.
static bool plan_launch(SweepParams& p, int pencils, int per_cta, int v, int nbi, int& grid, cudaStream_t s) {
  p.tiles_per_leaf = (pencils + per_cta - 1) / per_cta;
  p.n_items = p.nleaf * p.tiles_per_leaf;
  if (p.n_items <= 0) return false;
  p.div_tiles = FastDiv::make((unsigned)p.tiles_per_leaf);
  p.div_cb = FastDiv::make((unsigned)(p.b1 - p.b0));
  grid = p.n_items;
  if (kVariants[v].persistent && p.work) {
    cudaMemsetAsync(p.work, 0, sizeof(unsigned), s);
    grid = g_resident[nbi][v] < grid ? g_resident[nbi][v] : grid;
  } else {
    p.work = nullptr;
  }
  return true;
}

template <int NB, int P, int MINB>
static void launch_variant(const DevMesh& m, SweepParams p, int pencils, int v, cudaStream_t s) {
  constexpr int N = NB + 2 * kGhosts;
  int grid = 0;
  if (!plan_launch(p, pencils, P, v, nb_index(NB), grid, s)) return;
  switch (method_code(m.riemann, m.steepen, m.nf == 6)) {
    case 0: sweep_kernel<float, NB, P, MINB, 0><<<grid, N * P, sweep_smem<NB, P, 0>(), s>>>(m, p); break;
    case 1: sweep_kernel<float, NB, P, MINB, 1><<<grid, N * P, sweep_smem<NB, P, 1>(), s>>>(m, p); break;
    case 2: sweep_kernel<float, NB, P, MINB, 2><<<grid, N * P, sweep_smem<NB, P, 2>(), s>>>(m, p); break;
    case 3: sweep_kernel<float, NB, P, MINB, 3><<<grid, N * P, sweep_smem<NB, P, 3>(), s>>>(m, p); break;
    default: launch_sweep_de_f32<NB, P, MINB>(m, p, grid, s); break;   // dual energy (k_de_f32.cu)
  }
}

template <int NB, int CT, int MINB, int VEC>
static void launch_stream_variant(const DevMesh& m, SweepParams p, int pencils, int v, cudaStream_t s) {
  int grid = 0;
  if (!plan_launch(p, pencils, CT, v, nb_index(NB), grid, s)) return;
  constexpr size_t sh = stream_smem<CT, VEC>();
  if (m.nf == 6) {   // dual energy (k_de_f32.cu)
    launch_stream_de_f32<NB, CT, MINB, VEC>(m, p, grid, s);
    return;
  }
  switch (method_code(m.riemann, m.steepen)) {
    case 0: sweep_stream_kernel<float, NB, CT, MINB, VEC, 0><<<grid, CT, sh, s>>>(m, p); break;
    case 1: sweep_stream_kernel<float, NB, CT, MINB, VEC, 1><<<grid, CT, sh, s>>>(m, p); break;
    case 2: sweep_stream_kernel<float, NB, CT, MINB, VEC, 2><<<grid, CT, sh, s>>>(m, p); break;
    case 3: sweep_stream_kernel<float, NB, CT, MINB, VEC, 3><<<grid, CT, sh, s>>>(m, p); break;
  }
}

template <int NB>
static void prepare_nb(int sms) {
  prepare_variant<NB, 8, 3>(0, sms);
  prepare_variant<NB, 8, 4>(1, sms);
  prepare_variant<NB, 4, 6>(2, sms);
  prepare_variant<NB, 16, 1>(3, sms);
  prepare_variant<NB, 4, 8>(4, sms);
  prepare_variant<NB, 16, 2>(5, sms);
  prepare_stream_variant<NB, 64, 8, 0>(6, sms);
  prepare_stream_variant<NB, 128, 4, 0>(7, sms);
  prepare_stream_variant<NB, 64, 6, 0>(8, sms);
  prepare_stream_variant<NB, 32, 16, 0>(9, sms);
  prepare_stream_variant<NB, 64, 8, 3>(10, sms);
  prepare_stream_variant<NB, 64, 6, 3>(11, sms);
  for (int v = kNT; v < kNV; ++v) g_resident[nb_index(NB)][v] = g_resident[nb_index(NB)][v - kNT];
}

template <int NB>
static void launch_nb(const DevMesh& m, const SweepParams& p, int pencils, cudaStream_t s) {
  const int v = (p.variant >= 0 && p.variant < kNV) ? p.variant : 0;
  switch (v % kNT) {
    case 0: launch_variant<NB, 8, 3>(m, p, pencils, v, s); break;
    case 1: launch_variant<NB, 8, 4>(m, p, pencils, v, s); break;
    case 2: launch_variant<NB, 4, 6>(m, p, pencils, v, s); break;
    case 3: launch_variant<NB, 16, 1>(m, p, pencils, v, s); break;
    case 4: launch_variant<NB, 4, 8>(m, p, pencils, v, s); break;
    case 5: launch_variant<NB, 16, 2>(m, p, pencils, v, s); break;
    case 6: launch_stream_variant<NB, 64, 8, 0>(m, p, pencils, v, s); break;
    case 7: launch_stream_variant<NB, 128, 4, 0>(m, p, pencils, v, s); break;
    case 8: launch_stream_variant<NB, 64, 6, 0>(m, p, pencils, v, s); break;
    case 9: launch_stream_variant<NB, 32, 16, 0>(m, p, pencils, v, s); break;
    case 10: launch_stream_variant<NB, 64, 8, 3>(m, p, pencils, v, s); break;
    case 11: launch_stream_variant<NB, 64, 6, 3>(m, p, pencils, v, s); break;
  }
}

void launch_reduce_partials_f32(const DevMesh& m, const float* U, double* partials, int leaf0, int nleaf, int grid,
                                cudaStream_t s) {
  const int g = (grid > 0 && grid < nleaf) ? grid : nleaf;
  if (m.nf == 6) {
    switch (m.n) {
      case 8: reduce_partials_f32_kernel<8, 6><<<g, kReduceThreads, 0, s>>>(m, U, partials, leaf0, nleaf); break;
      case 16: reduce_partials_f32_kernel<16, 6><<<g, kReduceThreads, 0, s>>>(m, U, partials, leaf0, nleaf); break;
      case 32: reduce_partials_f32_kernel<32, 6><<<g, kReduceThreads, 0, s>>>(m, U, partials, leaf0, nleaf); break;
    }
    return;
  }
  switch (m.n) {
    case 8: reduce_partials_f32_kernel<8><<<g, kReduceThreads, 0, s>>>(m, U, partials, leaf0, nleaf); break;
    case 16: reduce_partials_f32_kernel<16><<<g, kReduceThreads, 0, s>>>(m, U, partials, leaf0, nleaf); break;
    case 32: reduce_partials_f32_kernel<32><<<g, kReduceThreads, 0, s>>>(m, U, partials, leaf0, nleaf); break;
  }
}

int sweep_variant_count_f32() { return kNV; }
SweepVariant sweep_variant_f32(int v) { return kVariants[v]; }

void launch_sweep_f32(const DevMesh& m, const SweepParams& p, int pencils, cudaStream_t s) {
  switch (m.n) {
    case 8: launch_nb<8>(m, p, pencils, s); break;
    case 16: launch_nb<16>(m, p, pencils, s); break;
    case 32: launch_nb<32>(m, p, pencils, s); break;
  }
}

template <int NB, int P>
static size_t adj_smem() {
  constexpr int N = NB + 2 * kGhosts;
  return sizeof(float) * (10 * N * (P + 1) + (NB + 1) * 40 * P);
}

template <int NB>
static void prepare_adj() {
  cudaFuncSetAttribute(adjoint_sweep_kernel<float, NB, kAdjPencils>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)adj_smem<NB, kAdjPencils>());
}

template <int NB>
static void adj_sweep_n(const DevMesh& m, const AdjSweepParams& p, cudaStream_t s) {
  constexpr int N = NB + 2 * kGhosts;
  adjoint_sweep_kernel<float, NB, kAdjPencils><<<p.n_items, N * kAdjPencils, adj_smem<NB, kAdjPencils>(), s>>>(m, p);
}

void launch_adjoint_sweep_f32(const DevMesh& m, const AdjSweepParams& p, cudaStream_t s) {
  if (p.n_items <= 0) return;
  switch (m.n) {
    case 8: adj_sweep_n<8>(m, p, s); break;
    case 16: adj_sweep_n<16>(m, p, s); break;
    case 32: adj_sweep_n<32>(m, p, s); break;
  }
}

void prepare_kernels_f32() {
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  prepare_nb<8>(sms);
  prepare_nb<16>(sms);
  prepare_nb<32>(sms);
  prepare_adj<8>();
  prepare_adj<16>();
  prepare_adj<32>();
}


}  // namespace cello
