// Once-per-device flags for host code.  A kernel's dynamic shared memory
// limit (cudaFuncSetAttribute) is a property of the kernel on one device, so
// a program that launches on several devices must opt in on each of them.
// No CUDA dependency: the logic is tested on the CPU.
#pragma once

#include <atomic>

namespace gatspi_host {

constexpr int kMaxDevices = 64;

// One flag per device, set once an action succeeded there.  Several host
// threads may call run() at once: on first use the action may then run more
// than once concurrently (it must be idempotent, as cudaFuncSetAttribute
// is), and it never runs again on a device after it succeeded.  Devices
// beyond kMaxDevices get no flag: the action runs on every call.
class PerDeviceOnce {
 public:
  // Returns 0 when the action already succeeded on `device`, else the
  // action's own result (0 = success, which sets the flag).
  template <class F>
  int run(int device, F&& action) {
    const bool tracked = device >= 0 && device < kMaxDevices;
    if (tracked && done_[device].load(std::memory_order_acquire)) return 0;
    const int rc = action();
    if (rc == 0 && tracked) done_[device].store(true, std::memory_order_release);
    return rc;
  }
  bool done(int device) const {
    return device >= 0 && device < kMaxDevices && done_[device].load(std::memory_order_acquire);
  }

 private:
  std::atomic<bool> done_[kMaxDevices] = {};
};

}  // namespace gatspi_host
