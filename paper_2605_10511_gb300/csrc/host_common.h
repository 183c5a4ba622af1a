// Host-side helpers shared by the library's C++ translation units.
#pragma once

#include <algorithm>
#include <cstdarg>
#include <cstdint>
#include <string>

#include "../../include/dpf.h"

namespace dpf {

// Records a printf-style message as this thread's last error and returns `st`.
dpf_status fail(dpf_status st, const char* fmt, ...);

// Number of worker threads for host-side loops (encoder, validation).
unsigned host_threads();

// Runs fn(i) for i in [0, n) over host_threads() threads.
template <class F>
void parallel_for(uint64_t n, F&& fn);

}  // namespace dpf

#include <thread>
#include <vector>

template <class F>
void dpf::parallel_for(uint64_t n, F&& fn) {
  const unsigned T = n < 2 ? 1u : (unsigned)std::min<uint64_t>(n, dpf::host_threads());
  if (T <= 1) {
    for (uint64_t i = 0; i < n; ++i) fn(i);
    return;
  }
  std::vector<std::thread> pool;
  pool.reserve(T);
  for (unsigned t = 0; t < T; ++t)
    pool.emplace_back([&, t] {
      for (uint64_t i = t; i < n; i += T) fn(i);
    });
  for (auto& th : pool) th.join();
}
