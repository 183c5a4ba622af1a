// Dimension scan + hash build (Kernel #1 of Sec. 3.1: scan, filter, build).
//
// The dimension's columns are decoded tile by tile with the same warp tiles
// as the fused kernel; rows passing the dimension predicates are either
// counted (first pass, sizes the table) or inserted (second pass) into an
// open-addressing table with linear probing.  A slot is one 64-bit word
// {key, payload} claimed with a single compare-and-swap; the payload packs
// the dictionary codes of up to two payload columns (16 bits each).
#include "tile.cuh"

namespace dpf {
namespace {

constexpr unsigned long long kEmptySlot = 0x0000000080000000ull;  // {INT32_MIN, 0}

template <bool kHost, bool kInsert>
__global__ void __launch_bounds__(256) build_kernel(const DevQuery* __restrict__ qdev, uint2* table,
                                                    uint32_t mask, unsigned long long* count,
                                                    unsigned int* status) {
  __shared__ __align__(16) DevQuery Q;
  {
    const uint4* src = reinterpret_cast<const uint4*>(qdev);
    uint4* dst = reinterpret_cast<uint4*>(&Q);
    for (uint32_t i = threadIdx.x; i < sizeof(DevQuery) / 16; i += blockDim.x) dst[i] = __ldg(src + i);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const uint64_t warp = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
  const uint64_t P = Q.page_rows;
  const uint64_t npages = (Q.nrows + P - 1) / P;
  const uint64_t tiles_per_page = (P / kMB + TB - 1) / TB;
  unsigned long long kept = 0;
  for (uint64_t w = warp; w < npages * tiles_per_page; w += nwarps) {
    const uint64_t p = w / tiles_per_page;
    const uint32_t i0 = uint32_t(w % tiles_per_page) * TB;
    const uint32_t prow = uint32_t(tmin<uint64_t>(P, Q.nrows - p * P));
    const uint32_t nmb_page = (prow + kMB - 1) / kMB;
    if (i0 >= nmb_page) continue;
    TileState T;
    tile_begin<kHost>(Q, p, i0, tmin<uint32_t>(TB, nmb_page - i0), lane, T);
    if (!tile_steps<kHost>(Q, T, nullptr, lane, status)) continue;
    if (!kInsert) {
      kept += __popc(T.alive);
      continue;
    }
    uint32_t key[TB][4], p0[TB][4], p1[TB][4], anym;
    MbHdr H[TB];
    tile_decode<kHost>(Q, Q.build_key, T, lane, key, anym, H, status);
    if (Q.build_npay > 0) tile_decode<kHost>(Q, Q.build_pay[0], T, lane, p0, anym, H, status);
    if (Q.build_npay > 1) tile_decode<kHost>(Q, Q.build_pay[1], T, lane, p1, anym, H, status);
#pragma unroll
    for (int t = 0; t < TB; ++t)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (!((T.alive >> (4 * t + k)) & 1u)) continue;
        const int32_t kv = int32_t(key[t][k]);
        if (kv == kEmptyKey) {
          atomicOr(status, S_CORRUPT);
          continue;
        }
        uint32_t pay = 0;
        if (Q.build_npay > 0) pay |= p0[t][k] & 0xffffu;
        if (Q.build_npay > 1) pay |= (p1[t][k] & 0xffffu) << 16;
        const unsigned long long slot = (unsigned long long)uint32_t(kv) | ((unsigned long long)pay << 32);
        uint32_t h = fmix32(uint32_t(kv)) & mask;
        bool done = false;
        for (uint32_t n = 0; n <= mask && !done; ++n) {
          unsigned long long* addr = reinterpret_cast<unsigned long long*>(table + h);
          const unsigned long long old = atomicCAS(addr, kEmptySlot, slot);
          if (old == kEmptySlot) {
            done = true;
          } else if (int32_t(uint32_t(old)) == kv) {
            atomicOr(status, S_DUPKEY);
            done = true;
          } else {
            h = (h + 1) & mask;
          }
        }
        if (!done) atomicOr(status, S_INTERNAL);
      }
  }
  if (!kInsert) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) kept += __shfl_down_sync(kFull, kept, d);
    if (lane == 0 && kept) atomicAdd(count, kept);
  }
}

__global__ void init_table_kernel(uint2* table, uint32_t slots) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < slots; i += gridDim.x * blockDim.x)
    reinterpret_cast<unsigned long long*>(table)[i] = kEmptySlot;
}

int build_grid(uint64_t nrows, uint64_t page_rows) {
  const uint64_t npages = (nrows + page_rows - 1) / page_rows;
  const uint64_t tiles = npages * ((page_rows / kMB + TB - 1) / TB);
  const uint64_t blocks = (tiles + 7) / 8;  // 8 warps per block
  return int(tmin<uint64_t>(tmax<uint64_t>(blocks, 1), 4096));
}

}  // namespace

cudaError_t launch_build_count(const BuildLaunch& L, cudaStream_t s) {
  const int g = build_grid(L.nrows, L.page_rows);
  if (L.host_data) build_kernel<true, false><<<g, 256, 0, s>>>(L.q, nullptr, 0, L.count, &L.sched->status);
  else build_kernel<false, false><<<g, 256, 0, s>>>(L.q, nullptr, 0, L.count, &L.sched->status);
  return cudaGetLastError();
}

cudaError_t launch_build_insert(const BuildLaunch& L, cudaStream_t s) {
  const int g = build_grid(L.nrows, L.page_rows);
  if (L.host_data) build_kernel<true, true><<<g, 256, 0, s>>>(L.q, L.table, L.mask, nullptr, &L.sched->status);
  else build_kernel<false, true><<<g, 256, 0, s>>>(L.q, L.table, L.mask, nullptr, &L.sched->status);
  return cudaGetLastError();
}

cudaError_t launch_init_table(uint2* table, uint32_t slots, cudaStream_t s) {
  const int g = int(tmin<uint32_t>((slots + 255) / 256, 2048u));
  init_table_kernel<<<g, 256, 0, s>>>(table, slots);
  return cudaGetLastError();
}

}  // namespace dpf
