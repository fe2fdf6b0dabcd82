// vbe_measure_fp64_rate: the FP64 pipe's instruction rate on this device,
// measured with a throughput kernel (the denominator of the float64
// workloads' ALU roofline).
//
// Each thread runs kChains independent dependency chains of one float64
// operation (fused multiply-add, add or multiply) for `iters` rounds, so the
// pipe, not the latency of a chain, bounds the kernel; a grid of several
// blocks per SM keeps every SM busy. The operands are chosen so that no
// value overflows, underflows or turns into a constant, and the results are
// written out, so no operation can be removed. The rate is the number of
// operations (warp lanes x chains x rounds) over the kernel's duration,
// timed with CUDA events on the caller's stream.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/vbe.h"

namespace {

constexpr int kChains = 8;
constexpr int kBlock = 256;

template <int OP>
__global__ void __launch_bounds__(kBlock) fp64_chains(int64_t iters, double a, double b, double* out) {
  double x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = 1.0 + (threadIdx.x + k) * 0x1p-30;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      if (OP == 0) x[k] = fma(x[k], a, b);   // x stays near b / (1 - a)
      else if (OP == 1) x[k] = x[k] + b;     // b tiny: grows by ulps
      else x[k] = x[k] * a;                  // a = 1 - 2^-40: decays slowly
    }
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int vbe_measure_fp64_rate(int32_t op, int64_t iters, double* out_per_s, double* scratch, void* stream) {
  if (!out_per_s || !scratch || iters <= 0 || op < 0 || op > 2) return VBE_ERR_INVALID;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return VBE_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return VBE_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const unsigned grid = (unsigned)sms * 8;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return VBE_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return VBE_ERR_CUDA;
  }
  const double a = 1.0 - 0x1p-40, b = 0x1p-60;
  cudaEventRecord(e0, s);
  if (op == 0) fp64_chains<0><<<grid, kBlock, 0, s>>>(iters, 0.5, 1.0, scratch);
  else if (op == 1) fp64_chains<1><<<grid, kBlock, 0, s>>>(iters, a, b, scratch);
  else fp64_chains<2><<<grid, kBlock, 0, s>>>(iters, a, b, scratch);
  cudaEventRecord(e1, s);
  int rc = VBE_OK;
  float ms = 0.f;
  if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
      cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f) {
    rc = VBE_ERR_CUDA;
  } else {
    const double ops = (double)grid * kBlock * kChains * (double)iters;
    *out_per_s = ops / (ms * 1e-3);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}
