// Measured FP32 issue rate of the device (cello_fp32_ffma_rate): the
// denominator of the sweep kernel's ALU roofline.  Not a step of the method.
#include "cello.h"
#include "cello_internal.h"

// Every thread runs kChains independent multiply-add chains (enough
// independent work to cover the pipeline latency at the launched occupancy),
// so the launch is bound by the FP32 pipes alone.
namespace cello {
namespace {

constexpr int kChains = 16;

__global__ void __launch_bounds__(256) ffma_rate_kernel(float* out, int iters, float a, float b) {
  float x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  // keeps the chains alive: the chains start non-negative and a, b > 0 keep
  // them so, so the store never happens (out may be null)
  if (s < 0.0f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace cello

extern "C" cello_status cello_fp32_ffma_rate(double* ffma_per_s, double* ms_out, void* stream) {
  using namespace cello;
  if (!ffma_per_s) return set_error(CELLO_EINVAL, "cello_fp32_ffma_rate: NULL argument");
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess || sms <= 0) return set_error(CELLO_ECUDA, "cello_fp32_ffma_rate: no usable device");
  const cudaStream_t s = (cudaStream_t)stream;
  const int threads = 256, blocks = sms * 8, iters = 1 << 14;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  float* out = nullptr;   // never written: the kernel's guard is never true
  e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  double best = 0.0, best_ms = 0.0;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {   // the first launch warms up
    cudaEventRecord(ev[0], s);
    ffma_rate_kernel<<<blocks, threads, 0, s>>>(out, iters, 0.999999f, 1e-7f);   // a, b > 0
    cudaEventRecord(ev[1], s);
    e = cudaEventSynchronize(ev[1]);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
    const double rate = (double)blocks * threads * kChains * iters / (ms * 1e-3);
    if (e == cudaSuccess && rep > 0 && rate > best) {
      best = rate;
      best_ms = ms;
    }
  }
  if (ev[0]) cudaEventDestroy(ev[0]);
  if (ev[1]) cudaEventDestroy(ev[1]);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(CELLO_ECUDA, cudaGetErrorString(e));
  *ffma_per_s = best;
  if (ms_out) *ms_out = best_ms;
  return CELLO_OK;
}
