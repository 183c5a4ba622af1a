// dpf_read_rate: the read bandwidth a kernel sees on a buffer in device
// memory or in mapped pinned host memory, measured the way the fused kernel
// reads compressed pages (16-byte read-only loads, every SM busy).  For
// host-resident tables it is the roofline denominator: the fused kernel's
// host-resident variant cannot read its pages faster than this (the paper's
// data path is bounded by the storage link the same way, Sec. 5).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "../../include/dpf.h"
#include "host_common.h"

namespace dpf {
std::recursive_mutex& ctx_mutex(dpf_ctx* c);
namespace {

// Grid-stride streaming read with four independent 16-byte loads in flight
// per thread; the XOR of everything read decides a store that never happens
// in practice but keeps the loads alive.
__global__ void __launch_bounds__(512) read_stream_kernel(const uint4* __restrict__ p, uint64_t n16,
                                                          unsigned int* sink) {
  uint4 a{0, 0, 0, 0};
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  for (; i + 3 * stride < n16; i += 4 * stride) {
    const uint4 v0 = __ldg(p + i), v1 = __ldg(p + i + stride), v2 = __ldg(p + i + 2 * stride),
                v3 = __ldg(p + i + 3 * stride);
    a.x ^= v0.x ^ v1.x ^ v2.x ^ v3.x;
    a.y ^= v0.y ^ v1.y ^ v2.y ^ v3.y;
    a.z ^= v0.z ^ v1.z ^ v2.z ^ v3.z;
    a.w ^= v0.w ^ v1.w ^ v2.w ^ v3.w;
  }
  for (; i < n16; i += stride) {
    const uint4 v = __ldg(p + i);
    a.x ^= v.x;
    a.y ^= v.y;
    a.z ^= v.z;
    a.w ^= v.w;
  }
  if ((a.x ^ a.y ^ a.z ^ a.w) == 0x5bd1e995u && a.x == 0x9e3779b9u) atomicAdd(sink, 1u);
}

}  // namespace
}  // namespace dpf

using namespace dpf;

extern "C" dpf_status dpf_read_rate(dpf_ctx* ctx, int32_t placement, uint64_t bytes, uint32_t reps, void* stream,
                                    double* gb_per_s) {
  if (!ctx || !gb_per_s) return fail(DPF_EINVAL, "NULL argument");
  if (placement != DPF_PLACE_DEVICE && placement != DPF_PLACE_HOST_PINNED)
    return fail(DPF_EINVAL, "placement %d", placement);
  if (bytes < (1u << 20) || bytes % 16 != 0 || bytes > (uint64_t(1) << 36))
    return fail(DPF_EINVAL, "bytes must be a multiple of 16 in [1 MiB, 64 GiB]");
  if (reps == 0) reps = 5;
  std::lock_guard<std::recursive_mutex> lk(ctx_mutex(ctx));
  int device = 0, prev = -1;
  dpf_status st = dpf_context_device(ctx, &device);
  if (st) return st;
  cudaGetDevice(&prev);
  if (prev != device) cudaSetDevice(device);
  struct Restore {
    int prev, dev;
    ~Restore() {
      if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    }
  } restore{prev, device};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void* host = nullptr;
  void* buf = nullptr;
  unsigned int* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto cleanup = [&] {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    if (placement == DPF_PLACE_DEVICE && buf) cudaFree(buf);
    if (host) cudaFreeHost(host);
  };
  cudaError_t e = cudaMalloc(&sink, sizeof(unsigned int));
  if (e == cudaSuccess && placement == DPF_PLACE_HOST_PINNED) {
    e = cudaHostAlloc(&host, bytes, cudaHostAllocMapped | cudaHostAllocPortable);
    if (e == cudaSuccess) {
      std::memset(host, 0x5a, bytes);  // touch every page
      e = cudaHostGetDevicePointer(&buf, host, 0);
    }
  } else if (e == cudaSuccess) {
    e = cudaMalloc(&buf, bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0x5a, bytes, s);
  }
  int sms = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const uint64_t n16 = bytes / 16;
  const int grid = sms * 4, block = 512;
  if (e == cudaSuccess) {
    read_stream_kernel<<<grid, block, 0, s>>>(static_cast<const uint4*>(buf), n16, sink);  // warm-up
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  for (uint32_t r = 0; r < reps && e == cudaSuccess; ++r) {
    read_stream_kernel<<<grid, block, 0, s>>>(static_cast<const uint4*>(buf), n16, sink);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cleanup();
  if (e != cudaSuccess) return fail(DPF_ECUDA, "dpf_read_rate: %s", cudaGetErrorString(e));
  *gb_per_s = double(bytes) * reps / (double(ms) * 1e-3) / 1e9;
  return DPF_OK;
}
