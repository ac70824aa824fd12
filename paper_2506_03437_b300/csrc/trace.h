// Host wall-clock trace of the runtime's phases.  With QK_TRACE set in the
// environment every mark prints one line to stderr:
//   qk-trace <call> <phase> <milliseconds since the previous mark>
// Device work is included only up to the call's last synchronisation.
#pragma once

#include <chrono>
#include <cstdio>
#include <cstdlib>

namespace qk {

inline bool trace_on() {
  static const bool on = std::getenv("QK_TRACE") != nullptr;
  return on;
}

struct Trace {
  const char* call;
  std::chrono::steady_clock::time_point t;
  explicit Trace(const char* c) : call(c), t(std::chrono::steady_clock::now()) {}
  void mark(const char* phase) {
    if (!trace_on()) return;
    auto now = std::chrono::steady_clock::now();
    std::fprintf(stderr, "qk-trace %s %s %.3f\n", call, phase,
                 std::chrono::duration<double, std::milli>(now - t).count());
    t = now;
  }
};

}  // namespace qk
