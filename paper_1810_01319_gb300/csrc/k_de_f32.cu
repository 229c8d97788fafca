// Float32 dual-energy sweeps (both forms with a sixth field rho e; method
// code RS | 4).  Compiled with the float32 sweep's flags; the planners in
// k_f32.cu compute the grid and call launch_sweep_de_f32 (shared-memory
// form) or launch_stream_de_f32 (register streaming).
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

// Register-streaming form: VEC = 3 stages three groups of four cells of the
// six fields per thread in shared memory, and the updated group.
template <int NB, int CT, int MINB, int VEC>
void launch_stream_de_f32(const DevMesh& m, const SweepParams& p, int grid, cudaStream_t s) {
  constexpr size_t sh = VEC == 3 ? sizeof(float4) * 4 * 6 * CT : 0;
  switch (method_code(m.riemann, m.steepen)) {
    case 0: sweep_stream_kernel<float, NB, CT, MINB, VEC, 4><<<grid, CT, sh, s>>>(m, p); break;
    case 1: sweep_stream_kernel<float, NB, CT, MINB, VEC, 5><<<grid, CT, sh, s>>>(m, p); break;
    case 2: sweep_stream_kernel<float, NB, CT, MINB, VEC, 6><<<grid, CT, sh, s>>>(m, p); break;
    case 3: sweep_stream_kernel<float, NB, CT, MINB, VEC, 7><<<grid, CT, sh, s>>>(m, p); break;
  }
}

// The streaming variants of the float32 table: {CTA size, min CTAs per SM, vector I/O}.
#define CELLO_DE_STREAM(X, NB) X(NB, 64, 8, 0) X(NB, 128, 4, 0) X(NB, 64, 6, 0) X(NB, 32, 16, 0) X(NB, 64, 8, 3) \
  X(NB, 64, 6, 3)
#define CELLO_DE_SINST(NB, CT, MINB, VEC) \
  template void launch_stream_de_f32<NB, CT, MINB, VEC>(const DevMesh&, const SweepParams&, int, cudaStream_t);
CELLO_DE_STREAM(CELLO_DE_SINST, 8)
CELLO_DE_STREAM(CELLO_DE_SINST, 16)
CELLO_DE_STREAM(CELLO_DE_SINST, 32)
#undef CELLO_DE_SINST
#undef CELLO_DE_STREAM

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
