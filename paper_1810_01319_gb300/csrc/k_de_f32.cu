// Float32 dual-energy sweeps (the shared-memory form with a sixth field rho
// e; method code RS | 4).  Compiled with the float32 sweep's flags; the
// planner in k_f32.cu computes the grid and calls launch_sweep_de_f32.
#include "kernels.cuh"

namespace cello {

template <int NB, int P, int RS>
static constexpr size_t de_smem() {
  return sizeof(float) * sweep_arrays(RS) * (NB + 2 * kGhosts) * P;
}

template <int NB, int P, int MINB>
void launch_sweep_de_f32(const DevMesh& m, const SweepParams& p, int grid, cudaStream_t s) {
  constexpr int T = (NB + 2 * kGhosts) * P;
  switch (method_code(m.riemann, m.steepen)) {
    case 0: sweep_kernel<float, NB, P, MINB, 4><<<grid, T, de_smem<NB, P, 4>(), s>>>(m, p); break;
    case 1: sweep_kernel<float, NB, P, MINB, 5><<<grid, T, de_smem<NB, P, 5>(), s>>>(m, p); break;
    case 2: sweep_kernel<float, NB, P, MINB, 6><<<grid, T, de_smem<NB, P, 6>(), s>>>(m, p); break;
    case 3: sweep_kernel<float, NB, P, MINB, 7><<<grid, T, de_smem<NB, P, 7>(), s>>>(m, p); break;
  }
}

template <int NB, int P, int MINB>
static void prepare_de() {
#define CELLO_DE_ATTR(RS)                                                                          \
  cudaFuncSetAttribute(sweep_kernel<float, NB, P, MINB, RS>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                       (int)de_smem<NB, P, RS>())
  CELLO_DE_ATTR(4);
  CELLO_DE_ATTR(5);
  CELLO_DE_ATTR(6);
  CELLO_DE_ATTR(7);
#undef CELLO_DE_ATTR
}

// The shared-memory variants of the float32 table: {pencils, min CTAs per SM}.
#define CELLO_DE_VARIANTS(X, NB) X(NB, 8, 3) X(NB, 8, 4) X(NB, 4, 6) X(NB, 16, 1) X(NB, 4, 8) X(NB, 16, 2)
#define CELLO_DE_INST(NB, P, MINB) \
  template void launch_sweep_de_f32<NB, P, MINB>(const DevMesh&, const SweepParams&, int, cudaStream_t);
CELLO_DE_VARIANTS(CELLO_DE_INST, 8)
CELLO_DE_VARIANTS(CELLO_DE_INST, 16)
CELLO_DE_VARIANTS(CELLO_DE_INST, 32)
#undef CELLO_DE_INST

void prepare_kernels_de_f32() {
#define CELLO_DE_PREP(NB, P, MINB) prepare_de<NB, P, MINB>();
  CELLO_DE_VARIANTS(CELLO_DE_PREP, 8)
  CELLO_DE_VARIANTS(CELLO_DE_PREP, 16)
  CELLO_DE_VARIANTS(CELLO_DE_PREP, 32)
#undef CELLO_DE_PREP
}
#undef CELLO_DE_VARIANTS

}  // namespace cello
