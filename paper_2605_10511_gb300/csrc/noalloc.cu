// dpf_execute_noalloc: one query through the fused kernel without any
// device allocation by the library during the call.
//
// Some callers cannot allocate device memory when they run a query: code
// running under a framework that has reserved all device memory in its own
// pool, latency-critical serving loops whose policy forbids allocation (an
// allocation can synchronise the device or fail under fragmentation), and
// callbacks that run inside another allocator.  For them the fused kernel's
// scratch (scheduler counters, the compiled plan, the per-group int64
// accumulators) lives in a fixed region of device memory that is part of
// the library image: the array below, reserved on every GPU that loads the
// library and held until the process exits.  The caller provides the
// output buffer.
#include <cstddef>
#include <mutex>

#include "../../include/dpf.h"
#include "dpf_internal.h"
#include "host_common.h"
#include "kernels.h"

namespace dpf {

dpf_status noalloc_compile(dpf_ctx* c, const dpf_plan* plan, DevQuery* Q, size_t* smem_tables, bool* host,
                           int* device, int* num_sms);
std::recursive_mutex& ctx_mutex(dpf_ctx* c);

// Capacity of the shared scratch region (1 MiB): scheduler state, the
// compiled plan and domain x (1 + aggregates) int64 accumulators.
constexpr size_t kNoAllocScratchBytes = DPF_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

constexpr size_t kOffSched = 0;
constexpr size_t kOffBegin = 256;
constexpr size_t kOffQuery = 512;
constexpr size_t kQueryBytes = (sizeof(DevQuery) + 255) / 256 * 256;
constexpr size_t kOffDone = kOffQuery + kQueryBytes;
constexpr size_t kOffAcc = kOffDone + 256;
// The header states the fixed part of the region in bytes; keep the two equal.
static_assert(kOffAcc == DPF_NOALLOC_FIXED_BYTES, "update DPF_NOALLOC_FIXED_BYTES in dpf.h");
static_assert(offsetof(Sched, status) % 4 == 0, "status word alignment");

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
uint8_t* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked
// up once per device (with that device current) and cached.
dpf_status scratch_address(int device, uint8_t** out) {
  if (device < 0 || device >= kMaxDevices) return fail(DPF_EINVAL, "device %d out of range", device);
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
      return fail(DPF_ECUDA, "cudaGetSymbolAddress(no-alloc scratch): %s", cudaGetErrorString(e));
    g_scratch_addr[device] = static_cast<uint8_t*>(p);
  }
  *out = g_scratch_addr[device];
  return DPF_OK;
}

}  // namespace
}  // namespace dpf

using namespace dpf;

extern "C" dpf_status dpf_execute_noalloc(dpf_ctx* ctx, const dpf_plan* plan, void* stream, dpf_record* out,
                                          uint64_t cap, uint32_t* out_count) {
  if (!ctx || !plan || !out || !out_count) return fail(DPF_EINVAL, "NULL argument");
  std::lock_guard<std::recursive_mutex> lk(ctx_mutex(ctx));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  {
    // The call copies its plan and ticket table from host stack memory; a
    // captured copy would keep the address of that dead frame and a replay
    // would launch the kernel on garbage, so a capturing stream is refused.
    cudaStreamCaptureStatus cap_st = cudaStreamCaptureStatusNone;
    const cudaError_t ce = cudaStreamIsCapturing(s, &cap_st);
    if (ce != cudaSuccess) return fail(DPF_ECUDA, "dpf_execute_noalloc: %s", cudaGetErrorString(ce));
    if (cap_st != cudaStreamCaptureStatusNone)
      return fail(DPF_EINVAL, "dpf_execute_noalloc cannot be captured into a CUDA graph (the stream is capturing)");
  }
  DevQuery Q;
  size_t smem_tables = 0;
  bool host = false;
  int device = 0, num_sms = 0;
  dpf_status st = noalloc_compile(ctx, plan, &Q, &smem_tables, &host, &device, &num_sms);
  if (st) return st;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != device) cudaSetDevice(device);
  struct Restore {
    int prev, dev;
    ~Restore() {
      if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    }
  } restore{prev, device};

  const uint64_t slots = uint64_t(Q.domain) * (1 + Q.naggs);
  const uint64_t need = kOffAcc + slots * 8;
  if (need > kNoAllocScratchBytes)
    return fail(DPF_EINVAL,
                "dpf_execute_noalloc: the plan needs %llu bytes of scratch (%llu groups x %u accumulators); "
                "the fixed region holds %llu bytes",
                (unsigned long long)need, (unsigned long long)Q.domain, 1 + Q.naggs,
                (unsigned long long)kNoAllocScratchBytes);
  if (cap < uint64_t(Q.domain ? Q.domain : 1))
    return fail(DPF_EINVAL, "dpf_execute_noalloc: out holds %llu records, the plan can produce %u",
                (unsigned long long)cap, Q.domain);
  uint8_t* base = nullptr;
  if ((st = scratch_address(device, &base))) return st;

  const uint32_t chunk_rows = kDefaultChunkRows;
  Q.chunk_rows = chunk_rows;
  Q.nchunks = (Q.nrows + chunk_rows - 1) / chunk_rows;
  Q.chunk_begin = 0;
  Q.use_smem_acc = slots <= kSmemAccSlots ? 1u : 0u;
  Q.acc = reinterpret_cast<unsigned long long*>(base + kOffAcc);
  Q.done = reinterpret_cast<unsigned int*>(base + kOffDone);
  Q.out = out;
  Q.out_n = out_count;
  const uint64_t qbegin[2] = {0, Q.nchunks};

  // the region keeps the previous call's contents: clear the counters and
  // accumulators, then write this call's plan
  cudaError_t e = cudaMemsetAsync(base + kOffSched, 0, sizeof(Sched), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(base + kOffDone, 0, 256 + slots * 8, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(base + kOffBegin, qbegin, sizeof qbegin, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(base + kOffQuery, &Q, sizeof Q, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return fail(DPF_ECUDA, "dpf_execute_noalloc: %s", cudaGetErrorString(e));

  FusedLaunch L{};
  L.queries = reinterpret_cast<const DevQuery*>(base + kOffQuery);
  L.qbegin = reinterpret_cast<const uint64_t*>(base + kOffBegin);
  L.nq = 1;
  L.total_chunks = Q.nchunks;
  L.sched = reinterpret_cast<Sched*>(base + kOffSched);
  L.threads = 256;
  L.smem_tables = smem_tables;
  L.acc_slots = Q.use_smem_acc ? uint32_t(slots) : 0u;
  L.host_data = host;
  L.text = needs_string_matcher(Q);
  L.min_blocks = kFusedMinBlocksLo;
  const int per_sm = fused_blocks_per_sm(L.threads, L.acc_slots, smem_tables, host, L.min_blocks);
  if (per_sm < 1) return fail(DPF_EINVAL, "dpf_execute_noalloc: fused kernel does not fit on an SM");
  L.grid = int(std::max<uint64_t>(1, std::min<uint64_t>(uint64_t(num_sms) * per_sm, Q.nchunks)));
  e = launch_fused(L, s);
  if (e != cudaSuccess) return fail(DPF_ECUDA, "dpf_execute_noalloc launch: %s", cudaGetErrorString(e));
  return DPF_OK;
}

extern "C" dpf_status dpf_noalloc_status(dpf_ctx* ctx, uint32_t* bits) {
  if (!ctx || !bits) return fail(DPF_EINVAL, "NULL argument");
  std::lock_guard<std::recursive_mutex> lk(ctx_mutex(ctx));
  int device = -1;
  dpf_status st = dpf_context_device(ctx, &device);
  if (st) return st;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != device) cudaSetDevice(device);
  struct Restore {
    int prev, dev;
    ~Restore() {
      if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    }
  } restore{prev, device};
  uint8_t* base = nullptr;
  if ((st = scratch_address(device, &base))) return st;
  uint32_t word = 0;
  const cudaError_t e = cudaMemcpy(&word, base + kOffSched + offsetof(Sched, status), sizeof word,
                                   cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(DPF_ECUDA, "dpf_noalloc_status: %s", cudaGetErrorString(e));
  *bits = word;
  if (word & S_CORRUPT)
    return fail(DPF_ECORRUPT, "the last dpf_execute_noalloc kernel met corrupt data (status 0x%x)", word);
  if (word & (S_INTERNAL | S_TIMEOUT))
    return fail(DPF_EINTERNAL, "the last dpf_execute_noalloc kernel hit a device invariant (status 0x%x)", word);
  return DPF_OK;
}
