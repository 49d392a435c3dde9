// FP64 FMA throughput probe behind lx3c_fp64_rate (include/lx3c.h): the
// measured denominator of the FP64 roofline that every integral class is
// bound by.  Each thread runs sixteen independent FMA chains so the FP64 pipe,
// not the 4-cycle dependent-issue latency, sets the rate; the grid fills
// every SM at the kernel's full occupancy.
#include <cuda_runtime.h>

#include <string>

#include "../../include/lx3c.h"

namespace lx3c {
void set_last_error(const std::string& msg);
}

namespace {

constexpr int kRateThreads = 512;
constexpr int kRateChains = 16;

__global__ void __launch_bounds__(kRateThreads) fp64_rate_kernel(long long iters, double b, double c,
                                                                  double* __restrict__ sink) {
  double a[kRateChains];
#pragma unroll
  for (int i = 0; i < kRateChains; ++i) a[i] = 1e-3 * threadIdx.x + i;
#pragma unroll 4
  for (long long it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kRateChains; ++i) a[i] = fma(a[i], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < kRateChains; ++i) s += a[i];
  // never true for these inputs; keeps every chain live
  if (s == -1.0) sink[blockIdx.x] = s;
}

}  // namespace

extern "C" lx3c_status lx3c_fp64_rate(int64_t iters, double* gflops, double* ms, void* stream) {
  if (!gflops || iters < 1) {
    lx3c::set_last_error("fp64_rate: bad argument");
    return LX3C_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, nsm = 0, per_sm = 0;
  double* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fp64_rate_kernel, kRateThreads, 0);
  const int grid = nsm * (per_sm > 0 ? per_sm : 1);
  if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(double) * grid);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float t = 0.0f;
  if (e == cudaSuccess) {
    const double b = 1.0 - 1e-13, c = 1e-7;
    fp64_rate_kernel<<<grid, kRateThreads, 0, st>>>(iters / 8 + 1, b, c, sink);  // warm-up
    cudaEventRecord(e0, st);
    fp64_rate_kernel<<<grid, kRateThreads, 0, st>>>(iters, b, c, sink);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  if (e != cudaSuccess) {
    lx3c::set_last_error(std::string("fp64_rate: ") + cudaGetErrorString(e));
    return LX3C_ECUDA;
  }
  const double flops = 2.0 * kRateChains * (double)iters * kRateThreads * grid;
  *gflops = flops / (t * 1e-3) / 1e9;
  if (ms) *ms = t;
  return LX3C_OK;
}
