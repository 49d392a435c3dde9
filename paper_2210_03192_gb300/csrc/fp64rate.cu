// FP64 FMA throughput probe behind lx3c_fp64_rate (include/lx3c.h): the
// measured denominator of the FP64 roofline that every integral class is
// bound by.  The grid fills every SM at the kernel's full occupancy.
#include <cuda_runtime.h>

#include <string>

#include "../../include/lx3c.h"

namespace lx3c {
void set_last_error(const std::string& msg);
}

namespace {

constexpr int kRateThreads = 256;

// Each thread keeps an 8 x 8 block of accumulators and, per step, reads 8 + 8
// operands from shared memory (broadcast) for 64 independent FMAs: the
// register-blocked outer product of a DGEMM, so that the FP64 pipe and not
// operand delivery sets the rate.
__global__ void __launch_bounds__(kRateThreads) fp64_rate_kernel(long long iters, double* __restrict__ sink) {
  __shared__ double sa[64], sb[64];
  if (threadIdx.x < 64) {
    sa[threadIdx.x] = 1.0 + 1e-3 * threadIdx.x;
    sb[threadIdx.x] = 1e-9 * (threadIdx.x + 1);
  }
  __syncthreads();
  double acc[8][8];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = 1e-3 * (r + c);
  const int o = (threadIdx.x >> 4) & 7;
  for (long long it = 0; it < iters; ++it) {
    const int q = (int)(it & 7);
    double a[8], b[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) a[r] = sa[(q * 8 + r + o) & 63];
#pragma unroll
    for (int c = 0; c < 8; ++c) b[c] = sb[(q * 8 + c) & 63];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[r][c] = fma(a[r], b[c], acc[r][c]);
  }
  double s = 0.0;
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) s += acc[r][c];
  // never true for these inputs; keeps every accumulator live
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
    fp64_rate_kernel<<<grid, kRateThreads, 0, st>>>(iters / 8 + 1, sink);  // warm-up
    cudaEventRecord(e0, st);
    fp64_rate_kernel<<<grid, kRateThreads, 0, st>>>(iters, sink);
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
  const double flops = 2.0 * 64.0 * (double)iters * kRateThreads * grid;
  *gflops = flops / (t * 1e-3) / 1e9;
  if (ms) *ms = t;
  return LX3C_OK;
}
