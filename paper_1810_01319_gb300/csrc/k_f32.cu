// Float32 PPM sweep (bulk arithmetic in float32, FMA contraction allowed).
#include "kernels.cuh"
#include "adjoint_kernels.cuh"

namespace cello {

template <int NB, int P>
static void sweep_f32_n(const DevMesh& m, const SweepParams& p, cudaStream_t s) {
  constexpr int N = NB + 2 * kGhosts;
  const size_t smem = sizeof(float) * 21 * N * P;
  auto k = sweep_kernel<float, NB, P>;
  const int grid = p.n_items;
  k<<<grid, N * P, smem, s>>>(m, p);
}

template <int NB, int P>
static void prepare_n() {
  constexpr int N = NB + 2 * kGhosts;
  cudaFuncSetAttribute(sweep_kernel<float, NB, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)(sizeof(float) * 21 * N * P));
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
  prepare_adj<8>();
  prepare_adj<16>();
  prepare_adj<32>();
  prepare_n<8, kPencilsPerTile>();
  prepare_n<16, kPencilsPerTile>();
  prepare_n<32, kPencilsPerTile>();
}

void launch_sweep_f32(const DevMesh& m, const SweepParams& p, int pencils, cudaStream_t s) {
  (void)pencils;
  if (p.n_items <= 0) return;
  switch (m.n) {
    case 8: sweep_f32_n<8, kPencilsPerTile>(m, p, s); break;
    case 16: sweep_f32_n<16, kPencilsPerTile>(m, p, s); break;
    case 32: sweep_f32_n<32, kPencilsPerTile>(m, p, s); break;
  }
}

}  // namespace cello
