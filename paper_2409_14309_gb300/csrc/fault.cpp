// Host-side fault injection (see fault.h).
#include "fault.h"

#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <mutex>

namespace sns {

namespace {
std::mutex g_mu;
int g_kind = kFaultNone;        // guarded by g_mu
long long g_left = 0;           // occurrences before the fault fires (guarded by g_mu)
bool g_explicit = false;        // set by fault_arm: the environment no longer applies
std::atomic<int> g_kind_fast{kFaultNone};   // g_kind, read without the lock
std::once_flag g_env_once;

sns_status parse(const char* spec, int* kind, long long* nth) {
  *kind = kFaultNone;
  *nth = 0;
  if (!spec || !*spec || strcmp(spec, "none") == 0) return SNS_OK;
  const char* colon = strchr(spec, ':');
  const size_t len = colon ? (size_t)(colon - spec) : strlen(spec);
  int k = kFaultNone;
  if (len == 5 && strncmp(spec, "alloc", 5) == 0) k = kFaultAlloc;
  else if (len == 6 && strncmp(spec, "launch", 6) == 0) k = kFaultLaunch;
  else if (len == 7 && strncmp(spec, "timeout", 7) == 0) k = kFaultTimeout;
  else return SNS_EINVAL;
  long long n = 1;
  if (colon) {
    char* end = nullptr;
    n = strtoll(colon + 1, &end, 10);
    if (end == colon + 1 || *end != '\0' || n < 1) return SNS_EINVAL;
  }
  *kind = k;
  *nth = n;
  return SNS_OK;
}

// SNSOLVE_FAULT is read once, at the first check; an unparsable value arms nothing.
void read_env() {
  std::call_once(g_env_once, [] {
    int k;
    long long n;
    if (parse(getenv("SNSOLVE_FAULT"), &k, &n) != SNS_OK) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_explicit) return;
    g_kind = k;
    g_left = n;
    g_kind_fast.store(k, std::memory_order_release);
  });
}
}  // namespace

bool fault_hit(FaultKind k) {
  read_env();
  if (g_kind_fast.load(std::memory_order_acquire) != k) return false;   // the common, unarmed case
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_kind != k) return false;
  if (--g_left > 0) return false;
  g_kind = kFaultNone;
  g_left = 0;
  g_kind_fast.store(kFaultNone, std::memory_order_release);
  return true;
}

sns_status fault_arm(const char* spec) {
  int k;
  long long n;
  const sns_status s = parse(spec, &k, &n);
  if (s != SNS_OK) return s;
  read_env();
  std::lock_guard<std::mutex> lk(g_mu);
  g_explicit = true;
  g_kind = k;
  g_left = n;
  g_kind_fast.store(k, std::memory_order_release);
  return SNS_OK;
}

int fault_armed(long long* left) {
  read_env();
  std::lock_guard<std::mutex> lk(g_mu);
  if (left) *left = g_left;
  return g_kind;
}

}  // namespace sns
