// probe.cu - measured FP64 FMA throughput of the current device: the
// denominator of the ALU roofline of FP64 trees (whose transcendental and
// division sequences run on the FP64 pipe, far slower than HBM on GB300).
//
// Every thread runs NACC independent FMA chains for `iters` steps, so the
// pipe, not the latency of one chain, sets the pace; one CTA of 256 threads
// per SM times the occupancy. The result is the FMA count times 2 (flops)
// over the CUDA-event time of the launch.
#include <cuda_runtime.h>

#include "fx/bulk.cuh"
#include "fx/runtime.hpp"

namespace fx {
namespace {

constexpr int kAcc = 8;

__global__ void __launch_bounds__(256) k_fp64_fma(double* out, int iters, double a, double b) {
  double acc[kAcc];
#pragma unroll
  for (int k = 0; k < kAcc; ++k) acc[k] = double(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kAcc; ++k) acc[k] = fma(acc[k], a, b);
  }
  double s = 0;
#pragma unroll
  for (int k = 0; k < kAcc; ++k) s += acc[k];
  if (s == 12345.678) out[blockIdx.x] = s;  // keeps the chains live; never true for a, b below
}

// One warp waits on an mbarrier that nothing arrives on, with a short poll
// limit: every lane must give up and record the timeout, and the kernel
// must finish (the failure path of the pipelines' bounded waits).
__global__ void k_wait_timeout(unsigned int* err, uint32_t polls) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    tma::mbar_init(&bar, 1);
    tma::fence_mbar_init();
  }
  __syncwarp();
  tma::wait(&bar, 0, err, polls);
}

}  // namespace
}  // namespace fx

using namespace fx;

extern "C" fx_status fx_selftest_wait_timeout(void* stream, unsigned int* word) {
  if (!word) return fail(FX_E_ARG, "null output");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned int* err = nullptr;
  FX_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&err), sizeof(unsigned int), st));
  FX_CUDA(cudaMemsetAsync(err, 0, sizeof(unsigned int), st));
  k_wait_timeout<<<1, 32, 0, st>>>(err, 1000);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(word, err, sizeof(unsigned int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(err, st);
  if (e != cudaSuccess) return cuda_fail(e, "wait-timeout self-test");
  return FX_OK;
}

extern "C" fx_status fx_fp64_fma_rate(void* stream, double* flops_per_s) {
  if (!flops_per_s) return fail(FX_E_ARG, "null output");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0, occ = 0;
  FX_CUDA(cudaGetDevice(&dev));
  FX_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  FX_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fp64_fma, 256, 0));
  if (occ < 1) occ = 1;
  const int grid = sms * occ, iters = 4096;
  double* out = nullptr;
  FX_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&out), sizeof(double) * grid, st));
  cudaEvent_t a, b;
  FX_CUDA(cudaEventCreate(&a));
  FX_CUDA(cudaEventCreate(&b));
  // a = 1 - 2^-30 and b = 2^-30 keep every chain bounded and never hit the sentinel
  const double ca = 1.0 - 9.313225746154785e-10, cb = 9.313225746154785e-10;
  k_fp64_fma<<<grid, 256, 0, st>>>(out, iters, ca, cb);  // warm-up
  cudaEventRecord(a, st);
  k_fp64_fma<<<grid, 256, 0, st>>>(out, iters, ca, cb);
  cudaEventRecord(b, st);
  cudaError_t e = cudaEventSynchronize(b);
  float ms = 0;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFreeAsync(out, st);
  if (e != cudaSuccess) return cuda_fail(e, "fp64 fma probe");
  const double fmas = double(grid) * 256.0 * kAcc * iters;
  *flops_per_s = 2.0 * fmas / (double(ms) * 1e-3);
  return FX_OK;
}
