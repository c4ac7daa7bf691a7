// Entry points whose implementation is pending: they validate nothing and
// return SNS_EINVAL so that callers fail loudly.
#include "snsolve.h"

extern "C" {
sns_status snsolve_server_create(sns_server** s, sns_ctx*, size_t, int) { if (s) *s = nullptr; return SNS_EINVAL; }
void snsolve_server_destroy(sns_server*) {}
sns_status snsolve_submit(sns_server*, const sns_problem*, const sns_opts*, double*, uint64_t*) { return SNS_EINVAL; }
sns_status snsolve_poll(sns_server*, uint64_t, int64_t, sns_info*) { return SNS_EINVAL; }
}
