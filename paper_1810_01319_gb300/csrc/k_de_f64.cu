// Float64 dual-energy sweeps (the shared-memory form with a sixth field rho
// e; method code RS | 4), built without FMA contraction like the float64
// sweep; k_f64.cu plans the launch and calls launch_sweep_de_f64.
#include "kernels.cuh"

namespace cello {

template <int NB, int RS>
static constexpr size_t de_smem64() {
  return sizeof(double) * sweep_arrays(RS) * (NB + 2 * kGhosts) * 8;
}

template <int NB>
void launch_sweep_de_f64(const DevMesh& m, const SweepParams& p, int grid, cudaStream_t s) {
  constexpr int T = (NB + 2 * kGhosts) * 8;
  switch (method_code(m.riemann, m.steepen)) {
    case 0: sweep_kernel<double, NB, 8, 2, 4><<<grid, T, de_smem64<NB, 4>(), s>>>(m, p); break;
    case 1: sweep_kernel<double, NB, 8, 2, 5><<<grid, T, de_smem64<NB, 5>(), s>>>(m, p); break;
    case 2: sweep_kernel<double, NB, 8, 2, 6><<<grid, T, de_smem64<NB, 6>(), s>>>(m, p); break;
    case 3: sweep_kernel<double, NB, 8, 2, 7><<<grid, T, de_smem64<NB, 7>(), s>>>(m, p); break;
  }
}

template void launch_sweep_de_f64<8>(const DevMesh&, const SweepParams&, int, cudaStream_t);
template void launch_sweep_de_f64<16>(const DevMesh&, const SweepParams&, int, cudaStream_t);
template void launch_sweep_de_f64<32>(const DevMesh&, const SweepParams&, int, cudaStream_t);

template <int NB>
static void prepare_de64() {
#define CELLO_DE_ATTR(RS)                                                                           \
  cudaFuncSetAttribute(sweep_kernel<double, NB, 8, 2, RS>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                       (int)de_smem64<NB, RS>())
  CELLO_DE_ATTR(4);
  CELLO_DE_ATTR(5);
  CELLO_DE_ATTR(6);
  CELLO_DE_ATTR(7);
#undef CELLO_DE_ATTR
}

void prepare_kernels_de_f64() {
  prepare_de64<8>();
  prepare_de64<16>();
  prepare_de64<32>();
}

}  // namespace cello
