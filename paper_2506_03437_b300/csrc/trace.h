// Host trace of the runtime's phases.
//  - Every traced call is an NVTX range named after the call, and every mark
//    an NVTX mark named after the phase that just ended, so a profiler that
//    records NVTX shows the call and its phases beside the kernels they
//    launched.  NVTX costs nothing when no such tool is attached.
//  - With QK_TRACE set in the environment every mark also prints one line to
//    stderr:  qk-trace <call> <phase> <milliseconds since the previous mark>
//    Device work is included only up to the call's last synchronisation.
#pragma once

#include <nvtx3/nvToolsExt.h>

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
  explicit Trace(const char* c) : call(c), t(std::chrono::steady_clock::now()) { nvtxRangePushA(c); }
  Trace(const Trace&) = delete;
  ~Trace() { nvtxRangePop(); }
  void mark(const char* phase) {
    nvtxMarkA(phase);
    if (!trace_on()) return;
    auto now = std::chrono::steady_clock::now();
    std::fprintf(stderr, "qk-trace %s %s %.3f\n", call, phase,
                 std::chrono::duration<double, std::milli>(now - t).count());
    t = now;
  }
};

}  // namespace qk
