// Error reporting, status strings and launch accounting.
#include <cstdarg>
#include <cstdio>

#include "hg_internal.h"

namespace {
thread_local char g_msg[512] = "";
std::atomic<int64_t> g_launches{0};
}  // namespace

namespace hg {
void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
    va_end(ap);
}
void note_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace hg

extern "C" const char *hg_last_error(void) { return g_msg; }

extern "C" int32_t hg_version(void) { return 10000; }

extern "C" int64_t hg_launch_count(void) { return g_launches.load(); }

extern "C" const char *hg_status_str(hg_status s) {
    switch (s) {
    case HG_OK: return "ok";
    case HG_EINVAL: return "invalid argument";
    case HG_ENOMEM: return "out of memory";
    case HG_ECUDA: return "CUDA error";
    case HG_EOVERFLOW: return "capacity exceeded";
    case HG_ESTEPLIMIT: return "step limit reached";
    case HG_ELOST: return "ray lost";
    case HG_EFORMAT: return "grid description invalid";
    case HG_EBADINPUT: return "bad ray input";
    case HG_ENOTFOUND: return "not found";
    }
    return "unknown status";
}

extern "C" hg_status hg_status_from_bits(uint32_t bits) {
    if (bits & HG_RAY_LOST) return HG_ELOST;
    if (bits & HG_RAY_STEPLIMIT) return HG_ESTEPLIMIT;
    if (bits & HG_RAY_OVERFLOW) return HG_EOVERFLOW;
    if (bits & HG_RAY_BADINPUT) return HG_EBADINPUT;
    return HG_OK;
}
