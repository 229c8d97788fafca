// Allocation-free variant of the CFL dt / conserved-totals reduction.
//
// cello_reduce keeps its per-leaf partial sums in device memory that the
// library cudaMalloc'ed when the mesh was built.  Some callers cannot let a
// library allocate at the point of use: code running inside a CUDA stream
// capture that must stay allocation-free, hosts with a fixed device-memory
// budget that hand every byte out up front, or embedding runtimes whose own
// allocator owns the device.  cello_reduce_noalloc serves them: its scratch
// is a fixed file-scope __device__ array that is part of the loaded module.
#include <mutex>

#include "cello.h"
#include "cello_internal.h"

namespace {

// Six doubles per leaf (dt candidate minimum and five field sums).  Every GPU
// that loads this library holds this array (1.5 MiB) until the process exits.
constexpr int kNoAllocMaxLeaves = 32768;
static __device__ __align__(256) double g_reduce_scratch[kNoAllocMaxLeaves * 6];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

}  // namespace

extern "C" cello_status cello_reduce_noalloc(cello_mesh* mesh, const void* U, double cfl, double* dt_next_dev,
                                             double* totals_dev, void* stream) {
  using namespace cello;
  if (!mesh || !U) return set_error(CELLO_EINVAL, "cello_reduce_noalloc: NULL argument");
  if ((reinterpret_cast<uintptr_t>(U) & 255u) != 0)
    return set_error(CELLO_EINVAL, "cello_reduce_noalloc: U is not 256-byte aligned");
  const DevMesh dm = mesh_dev(mesh);
  if (dm.B > kNoAllocMaxLeaves)
    return set_error(CELLO_EINVAL, "cello_reduce_noalloc: the mesh has more leaves than the fixed scratch holds "
                                   "(at most 32768); use cello_reduce");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return set_error(CELLO_ECUDA, "cello_reduce_noalloc: no usable current device");
  double* scratch = nullptr;
  {
    // one-time set-up per device, with that device current: the device
    // address of the file-scope array (its host-side name is only a stand-in)
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
      double* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress((void**)&p, g_reduce_scratch);
      if (e != cudaSuccess) return set_error(CELLO_ECUDA, cudaGetErrorString(e));
      g_scratch_ptr[dev] = p;
    }
    scratch = g_scratch_ptr[dev];
  }
  launch_reduce(dm, U, mesh_precision(mesh), cfl, scratch, dt_next_dev, totals_dev, (cudaStream_t)stream);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(CELLO_ECUDA, cudaGetErrorString(e));
  return CELLO_OK;
}
