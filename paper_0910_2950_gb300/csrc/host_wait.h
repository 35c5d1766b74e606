// Bounded host waits.  Plain C++ with no CUDA types, so the polling logic is
// compiled and tested on its own on a CPU (the runtime feeds it
// cudaStreamQuery / cudaEventQuery).
#pragma once

namespace fg {

enum WaitResult { WAIT_DONE = 0, WAIT_ERROR = 1, WAIT_TIMEOUT = 2 };

// Polls query() -- 0: finished, 1: still running, anything else: error --
// until the work has finished or failed, or until more than limit_s seconds
// of now() have passed since the first poll.  Between polls it calls
// pause(us) with a pause that doubles from 2 us up to 1 ms, so short waits
// stay responsive and long ones cost little host time.
template <class Query, class Now, class Pause>
WaitResult wait_limited(Query query, Now now, Pause pause, double limit_s) {
  const double t0 = now();
  double us = 2.0;
  for (;;) {
    const int q = query();
    if (q == 0) return WAIT_DONE;
    if (q != 1) return WAIT_ERROR;
    if (now() - t0 > limit_s) return WAIT_TIMEOUT;
    pause(us);
    us = us < 500.0 ? 2.0 * us : 1000.0;
  }
}

}  // namespace fg
