// vbe_reduce_add_f64_noalloc: the full float64 sum reduction without any
// device allocation.
//
// The executor's full-reduction kernels keep block partials and a
// completion counter in scratch memory that the library allocates. Some
// callers cannot let a library allocate device memory on their hot path:
// code whose stream work is being captured into a CUDA graph by someone
// else, plugin "enqueue" functions of inference engines that must not
// allocate, real-time loops that plan all memory up front. For them this
// entry point keeps its scratch in a fixed, file-scope device array that
// is part of the loaded library (every GPU that loads it holds the array
// until the process exits) and allocates nothing: the caller passes the
// input and the output, both in device memory.
//
// Set-up: the first call on a device looks up the device address of the
// array (cudaGetSymbolAddress, with that device current) and keeps it; make
// that first call before any stream capture. Every call shares the one
// array, so calls that overlap on the GPU (different streams, or several
// host threads) race and give wrong sums; serialise them.
//
// CUDA errors: an error already pending on the calling thread (left by
// earlier, unrelated work) is reported as VBE_ERR_CUDA before anything is
// enqueued and is left pending for its owner to read; an error of this
// call's own launch is reported as VBE_ERR_CUDA and cleared.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/vbe.h"

namespace {

constexpr int kBlock = 256;                  // threads per block
constexpr int64_t kChunk = 16384;            // elements summed into one partial
constexpr int64_t kMaxChunks = 65536;        // partials the scratch holds
constexpr int kMaxDevices = 64;

// partials (kMaxChunks doubles) followed by the completion counter
static __device__ __align__(256) unsigned char g_noalloc_scratch[kMaxChunks * 8 + 256];

void* g_scratch_addr[kMaxDevices];
std::mutex g_setup_mu;

__device__ double block_sum(double v) {
  __shared__ double sh[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  }
  __syncthreads();
  return v;
}

// One partial per fixed-size chunk (so the summation order depends only on
// n, not on the grid), then the last block to finish sums the partials in
// chunk order.
__global__ void __launch_bounds__(kBlock) sum_chunks(const double* __restrict__ x, int64_t n, int64_t nchunks,
                                                     double* __restrict__ out, unsigned char* scratch) {
  double* partials = reinterpret_cast<double*>(scratch);
  unsigned* counter = reinterpret_cast<unsigned*>(scratch + kMaxChunks * 8);
  __shared__ int s_last;
  for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int64_t lo = c * kChunk, hi = min(n, lo + kChunk);
    double acc = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += kBlock) acc += x[i];
    acc = block_sum(acc);
    if (threadIdx.x == 0) {
      partials[c] = acc;
      __threadfence();
      s_last = atomicAdd(counter, 1u) == (unsigned)(nchunks - 1);
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      double v = 0.0;
      const volatile double* pp = partials;
      for (int64_t i = threadIdx.x; i < nchunks; i += kBlock) v += pp[i];
      v = block_sum(v);
      if (threadIdx.x == 0) {
        *out = v;
        *counter = 0u;
      }
    }
    __syncthreads();
  }
}

}  // namespace

extern "C" int vbe_reduce_add_f64_noalloc(const double* x, int64_t n, double* out, void* stream) {
  if (n < 0 || out == nullptr || (n > 0 && x == nullptr)) return VBE_ERR_INVALID;
  if (n > kMaxChunks * kChunk) return VBE_ERR_INVALID;  // beyond the scratch: 2^30 elements
  // an earlier error belongs to someone else: report it, do not clear it
  if (cudaPeekAtLastError() != cudaSuccess) return VBE_ERR_CUDA;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return VBE_ERR_CUDA;
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev]) {
      // the array's name is a host-side stand-in; the kernel needs its
      // device address on this device
      if (cudaGetSymbolAddress(&g_scratch_addr[dev], g_noalloc_scratch) != cudaSuccess) {
        g_scratch_addr[dev] = nullptr;
        cudaGetLastError();
        return VBE_ERR_CUDA;
      }
    }
    scratch = g_scratch_addr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the completion counter must start at zero
  if (cudaMemsetAsync(static_cast<unsigned char*>(scratch) + kMaxChunks * 8, 0, sizeof(unsigned), s) !=
      cudaSuccess)
    return VBE_ERR_CUDA;
  const int64_t nchunks = n > 0 ? (n + kChunk - 1) / kChunk : 1;
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t grid = nchunks < 4LL * sms ? nchunks : 4LL * sms;
  sum_chunks<<<(unsigned)grid, kBlock, 0, s>>>(x, n, nchunks, out, static_cast<unsigned char*>(scratch));
  // nothing was pending before this call, so an error here is this launch's
  return cudaGetLastError() == cudaSuccess ? VBE_OK : VBE_ERR_CUDA;
}
