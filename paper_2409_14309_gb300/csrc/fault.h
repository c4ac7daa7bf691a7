// Host-side fault injection.  Nothing here touches the GPU: an armed fault
// makes one host-side check report a failure, so the error paths (status
// codes, skipped work, a context that stays usable) can be exercised without
// faulting, trapping or hanging a device.
//
// Spec "<kind>[:<n>]", from the environment variable SNSOLVE_FAULT (read once)
// or snsolve_debug_set_fault: the n-th occurrence (default 1) of <kind> fails,
// once, then the fault disarms.  Kinds:
//   alloc    one of the library's own allocations (context pinned buffer,
//            per-thread pinned buffer, server arena, batched staging) reports
//            SNS_ENOMEM without allocating;
//   launch   the check after a kernel launch reports SNS_ECUDA (the kernel
//            itself was launched and runs to completion);
//   timeout  the host's read of a device error word (sketch waits, QR polls)
//            reports an expired wait: SNS_ETIMEOUT.
#pragma once
#include "snsolve.h"

namespace sns {

enum FaultKind { kFaultNone = 0, kFaultAlloc = 1, kFaultLaunch = 2, kFaultTimeout = 3 };

// True exactly once: at the armed kind's n-th occurrence.
bool fault_hit(FaultKind k);
// Parses a spec; an empty or "none" spec disarms.  SNS_EINVAL on a bad spec.
sns_status fault_arm(const char* spec);
// Armed kind and occurrences left before it fires (kFaultNone, 0 when disarmed).
int fault_armed(long long* left);
// Records an injected failure as the thread's last error text and returns s.
sns_status record_injected(const char* what, sns_status s);

}  // namespace sns
