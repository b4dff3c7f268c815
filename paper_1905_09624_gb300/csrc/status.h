// Status and error message of the C ABI (CUDA-free: also used by the serve
// scheduler, which builds without the CUDA toolkit for host-only tests).
#pragma once
#include "cobs_gpu.h"

namespace cobs {

// Record a printf-style message for cobs_last_error() on this thread; returns s.
cobs_status set_error(cobs_status s, const char *fmt, ...);

}  // namespace cobs

namespace cobs {

// Host-side fault injection (cobs_debug_fail_alloc): true when the library's
// next device or pinned-host allocation must fail as if memory were exhausted.
bool alloc_injected_failure();

}  // namespace cobs

namespace cobs {

// cobs_debug_build_scratch: scratch budget of the device build's waves in bytes
// (0 = the library's choice).
uint64_t build_scratch_override();

}  // namespace cobs
