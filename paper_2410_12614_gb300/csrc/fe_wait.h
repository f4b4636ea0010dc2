// Decision rule of the kernels' bounded waits (mbarrier phases of the
// persistent tensor-core kernel), written once for the device code and for
// host-side tests of the rule.
//
// A wait gives up only when its own phase has made no progress for longer
// than the launch's limit, counted from the start of that wait: the limit
// bounds a stall, never the running time of a launch, so a launch of any
// length whose waits each complete in time never gives up.  Each probe of the
// barrier may suspend the waiting thread for at most the suspend hint, which
// never exceeds the limit.  The clock of a wait is read after its first
// unsuccessful probe (a wait satisfied at once reads no clock), so a stalled
// wait gives up between limit and limit + 2 hints (at most 3 limits) after it
// began.
#pragma once

#include <cstdint>

#if defined(__CUDACC__)
#define FE_WAIT_FN __host__ __device__ __forceinline__
#else
#define FE_WAIT_FN inline
#endif

namespace fe {

// Longest suspension of one try_wait probe (ns).
constexpr uint32_t kWaitSuspendNs = 100000;

FE_WAIT_FN uint32_t wait_suspend_hint(unsigned long long limit_ns) {
    return limit_ns < kWaitSuspendNs ? static_cast<uint32_t>(limit_ns) : kWaitSuspendNs;
}

// True once a wait that began at t_start (globaltimer, ns) and is still
// unsatisfied at t_now has exceeded limit_ns.
FE_WAIT_FN bool wait_expired(unsigned long long t_start, unsigned long long t_now, unsigned long long limit_ns) {
    return t_now - t_start > limit_ns;
}

}  // namespace fe
