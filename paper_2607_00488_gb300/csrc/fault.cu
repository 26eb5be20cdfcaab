// Host-side fault injection: exercises the library's failure paths (a device
// allocation that fails, a kernel launch that reports an error, a device wait
// that expires) without faulting, trapping or hanging the GPU.
//
//   alloc:   the selected device allocation is not made and reports
//            cudaErrorMemoryAllocation (the entry point returns SRW_ENOMEM);
//   launch:  the selected launch check reports cudaErrorLaunchFailure (the
//            entry point returns SRW_ECUDA; a graph being captured is dropped);
//   timeout: the selected fold launch makes one of its waits wait on an
//            mbarrier that nothing arrives on, with a 1 ms limit; the wait
//            gives up and the kernel takes the same abort path as a producer
//            that never delivers (status bit, NaN results for the affected
//            points, SRW_ETIMEOUT from host-pointer calls).
//
// A fault is armed by srw_fault_inject() or, once per process, by the
// environment variable SRW_FAULT = alloc | launch | timeout, optionally
// followed by ":N" to let N matching events pass first.  It fires once and
// disarms.

#include <cstdlib>
#include <cstring>
#include <mutex>

#include "srw_internal.h"

namespace srw {
namespace {

std::mutex g_fault_mutex;
int g_fault_kind = SRW_FAULT_NONE;
long long g_fault_skip = 0;
bool g_env_read = false;
thread_local bool g_timeout_fired = false;

// "kind" or "kind:N"; returns false on anything else.
bool parse_spec(const char* spec, int* kind, long long* skip) {
  if (spec == nullptr) return false;
  static const struct {
    const char* name;
    int kind;
  } names[] = {{"alloc", SRW_FAULT_ALLOC}, {"launch", SRW_FAULT_LAUNCH}, {"timeout", SRW_FAULT_TIMEOUT}};
  for (const auto& n : names) {
    const size_t len = std::strlen(n.name);
    if (std::strncmp(spec, n.name, len) != 0) continue;
    const char* rest = spec + len;
    if (*rest == '\0') {
      *kind = n.kind;
      *skip = 0;
      return true;
    }
    if (*rest != ':' || rest[1] == '\0') return false;
    char* end = nullptr;
    const long long v = std::strtoll(rest + 1, &end, 10);
    if (*end != '\0' || v < 0) return false;
    *kind = n.kind;
    *skip = v;
    return true;
  }
  return false;
}

void read_env_locked() {
  if (g_env_read) return;
  g_env_read = true;
  int kind = SRW_FAULT_NONE;
  long long skip = 0;
  if (parse_spec(std::getenv("SRW_FAULT"), &kind, &skip)) {
    g_fault_kind = kind;
    g_fault_skip = skip;
  }
}

}  // namespace

bool fault_fire(int kind) {
  std::lock_guard<std::mutex> lock(g_fault_mutex);
  read_env_locked();
  if (g_fault_kind != kind) return false;
  if (g_fault_skip > 0) {
    --g_fault_skip;
    return false;
  }
  g_fault_kind = SRW_FAULT_NONE;
  if (kind == SRW_FAULT_TIMEOUT) g_timeout_fired = true;
  return true;
}

bool fault_take_timeout_fired() {
  const bool f = g_timeout_fired;
  g_timeout_fired = false;
  return f;
}

}  // namespace srw

extern "C" srw_status srw_fault_inject(int kind, long long skip) {
  if (kind < SRW_FAULT_NONE || kind > SRW_FAULT_TIMEOUT || skip < 0) return SRW_EINVAL;
  std::lock_guard<std::mutex> lock(srw::g_fault_mutex);
  srw::g_env_read = true;  // an explicit setting overrides the environment
  srw::g_fault_kind = kind;
  srw::g_fault_skip = kind == SRW_FAULT_NONE ? 0 : skip;
  return SRW_OK;
}

extern "C" srw_status srw_fault_pending(int* kind) {
  if (kind == nullptr) return SRW_EINVAL;
  std::lock_guard<std::mutex> lock(srw::g_fault_mutex);
  srw::read_env_locked();
  *kind = srw::g_fault_kind;
  return SRW_OK;
}

extern "C" srw_status srw_fault_parse(const char* spec, int* kind, long long* skip) {
  int k = SRW_FAULT_NONE;
  long long s = 0;
  if (!srw::parse_spec(spec, &k, &s)) return SRW_EINVAL;
  if (kind) *kind = k;
  if (skip) *skip = s;
  return SRW_OK;
}
