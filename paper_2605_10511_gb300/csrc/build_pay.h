// Encoding of a hash build's payload sources shared by the planner
// (api.cpp) and the build kernel (build_hash.cu).
#pragma once
#include <cstdint>

namespace dpf {

// Q.build_pay[f] at or above this value takes payload field f from the
// group-id bits of the scan's survivor entries: {shift << 8 | bits}.
constexpr int32_t kPayFromGid = 0x40000000;

}  // namespace dpf
