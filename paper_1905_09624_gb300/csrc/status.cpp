// Thread-local error message behind cobs_last_error().
#include <cstdarg>
#include <cstdio>
#include <string>

#include "status.h"

namespace cobs {

static thread_local std::string g_err;

cobs_status set_error(cobs_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

}  // namespace cobs

extern "C" const char *cobs_last_error(void) { return cobs::g_err.c_str(); }

// ------------------------------------------------------- fault injection
#include <atomic>

namespace cobs {

// Allocations that may still succeed; negative = injection off.
static std::atomic<int64_t> g_alloc_left{-1};

bool alloc_injected_failure() {
    int64_t left = g_alloc_left.load();
    while (left > 0)
        if (g_alloc_left.compare_exchange_weak(left, left - 1)) return false;
    return left == 0;
}

}  // namespace cobs

extern "C" void cobs_debug_fail_alloc(int64_t after) { cobs::g_alloc_left.store(after < 0 ? -1 : after); }

// ------------------------------------------------- build wave budget
namespace cobs {

static std::atomic<uint64_t> g_build_scratch{0};

uint64_t build_scratch_override() { return g_build_scratch.load(); }

}  // namespace cobs

extern "C" void cobs_debug_build_scratch(uint64_t bytes) { cobs::g_build_scratch.store(bytes); }
