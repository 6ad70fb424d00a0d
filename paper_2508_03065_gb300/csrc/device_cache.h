// Per-device, thread-safe one-time launch set-up.
//
// A persistent kernel needs two things prepared once per GPU before its first
// launch there: its dynamic shared-memory limit (cudaFuncSetAttribute acts on
// the current device's context) and its grid size (SMs x resident CTAs, which
// depends on the device). PerDevice keeps one such value per device ordinal:
// the first caller for a device runs the set-up under a mutex, later callers
// read the stored value without locking. A failed set-up stores nothing, so
// the next call tries again. Plain C++ (no CUDA types), so that the logic is
// tested on the host.
#pragma once

#include <atomic>
#include <mutex>

namespace msrc {

constexpr int kMaxDevices = 64;

class PerDevice {
 public:
  // Value for device `dev` (0 <= dev < kMaxDevices): the stored one, or the
  // result of init(&value) run once, with a zero status, under the lock.
  // init returns a status (0 = success) and must set a value > 0 on success.
  // Returns init's status, or -1 for a device ordinal out of range.
  template <class Init>
  int get(int dev, Init&& init, int* out) {
    if (dev < 0 || dev >= kMaxDevices) return -1;
    int v = value_[dev].load(std::memory_order_acquire);
    if (v > 0) {
      *out = v;
      return 0;
    }
    std::lock_guard<std::mutex> lock(mutex_);
    v = value_[dev].load(std::memory_order_relaxed);
    if (v <= 0) {
      int fresh = 0;
      const int st = init(&fresh);
      if (st != 0) return st;
      if (fresh <= 0) return -2;
      v = fresh;
      value_[dev].store(v, std::memory_order_release);
    }
    *out = v;
    return 0;
  }

 private:
  std::atomic<int> value_[kMaxDevices] = {};
  std::mutex mutex_;
};

}  // namespace msrc
