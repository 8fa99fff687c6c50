// Diagnostics: the FP64 FMA rate of this GPU (pw_diag_fp64_fma_rate), measured by a kernel of
// independent FMA chains on every SM, so that DFMA-bound kernels have a measured roofline.
#include <algorithm>

#include "pw_internal.cuh"

namespace pw {
namespace {

constexpr int kChains = 8;       // independent FMA chains per thread (hides the FMA latency)
constexpr int kDiagThreads = 256;

// each thread runs kChains chains of `iters` dependent FMAs x <- x * a + b; the result is kept
// live through an output that is written only if it is not finite (never, for these values)
__global__ void __launch_bounds__(kDiagThreads) k_dfma_chains(int iters, double a, double b, double* sink) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  if (!isfinite(s)) sink[blockIdx.x] = s;
}

}  // namespace
}  // namespace pw

using namespace pw;

extern "C" PW_API int pw_diag_fp64_fma_rate(void* stream, double* tflops, double* ms) {
  if (!tflops) return set_error(PW_EINVAL, "NULL output");
  const cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, nsm = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dfma_chains, kDiagThreads, 0);
  if (e != cudaSuccess) return cuda_status(e, "FP64 rate set-up");
  const int grid = nsm * std::max(per_sm, 1);
  const int iters = 2048;
  double* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMalloc(&sink, sizeof(double) * grid);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // the first repetition warms up
    e = cudaEventRecord(e0, st);
    k_dfma_chains<<<grid, kDiagThreads, 0, st>>>(iters, 0.999999, 1e-7, sink); count_launch();
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (rep > 0) best = std::min(best, t);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  if (e != cudaSuccess) return cuda_status(e, "FP64 rate kernel");
  const double flops = 2.0 * (double)grid * kDiagThreads * iters * 16 * kChains;
  *tflops = flops / (best * 1e-3) / 1e12;
  if (ms) *ms = best;
  return PW_OK;
}
