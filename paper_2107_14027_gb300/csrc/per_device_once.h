// Once-per-device initialisation of a kernel's function attributes.
//
// cudaFuncSetAttribute (e.g. the dynamic shared memory limit of a kernel that
// needs more than the 48 KB default) applies to the context of the device
// that is current when it is called.  A launcher that remembered "done" in
// one process-wide flag would skip the call on every further device and its
// first launch there would fail.  PerDeviceOnce keeps one bit per device
// ordinal, set with an atomic OR after the call succeeded; host threads that
// race on the first launch may both make the (idempotent) call.  Ordinals at
// or beyond kBits are served by making the call every time.
//
// Header-only and free of CUDA types so that its logic can be checked on a
// host without a GPU (tests/cpp/per_device_once_test.cpp).
#pragma once

#include <atomic>
#include <cstdint>

namespace acmhd {

class PerDeviceOnce {
 public:
  static constexpr int kBits = 64;

  // get_device(int*) -> status, set() -> status; status 0 means success.
  // Returns the first non-zero status, or 0.
  template <class GetDevice, class Set>
  int run(GetDevice get_device, Set set) {
    int dev = 0;
    int st = static_cast<int>(get_device(&dev));
    if (st != 0) return st;
    const bool tracked = dev >= 0 && dev < kBits;
    const uint64_t bit = tracked ? (uint64_t(1) << dev) : 0;
    if (tracked && (done_.load(std::memory_order_acquire) & bit)) return 0;
    st = static_cast<int>(set());
    if (st == 0 && tracked) done_.fetch_or(bit, std::memory_order_acq_rel);
    return st;
  }

 private:
  std::atomic<uint64_t> done_{0};
};

}  // namespace acmhd
