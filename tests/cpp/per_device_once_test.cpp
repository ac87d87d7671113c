// Host-only check of PerDeviceOnce (paper_2107_14027_gb300/csrc/
// per_device_once.h): the set-up call runs once per device ordinal, again
// after a failure, every time for ordinals beyond the tracked range, and not
// at all when the device query fails.  Prints "ok" and exits 0 on success.
#include <cstdio>
#include <thread>
#include <vector>

#include "per_device_once.h"

static int fail(const char* what) {
  std::printf("FAIL: %s\n", what);
  return 1;
}

int main() {
  acmhd::PerDeviceOnce once;
  int current = 0, calls[128] = {};
  auto get = [&](int* d) { *d = current; return 0; };
  auto set = [&] { ++calls[current]; return 0; };

  // first launch on device 0, then on device 1, then back on both
  for (int dev : {0, 0, 1, 1, 0, 1, 3}) {
    current = dev;
    if (once.run(get, set) != 0) return fail("status");
  }
  if (calls[0] != 1 || calls[1] != 1 || calls[3] != 1) return fail("once per device");

  // a failed set-up is retried on the next launch
  current = 5;
  int attempts = 0;
  if (once.run(get, [&] { ++attempts; return 7; }) != 7) return fail("error passed on");
  if (once.run(get, [&] { ++attempts; return 0; }) != 0) return fail("retry");
  if (once.run(get, [&] { ++attempts; return 0; }) != 0) return fail("after retry");
  if (attempts != 2) return fail("retry count");

  // ordinals beyond the tracked range: called every time
  current = 100;
  for (int i = 0; i < 3; ++i) once.run(get, set);
  if (calls[100] != 3) return fail("untracked ordinal");

  // the device query fails: nothing is set up, its status is returned
  int never = 0;
  if (once.run([](int*) { return 9; }, [&] { ++never; return 0; }) != 9 || never != 0)
    return fail("device query error");

  // concurrent first launches on one device: at least one call, all succeed
  acmhd::PerDeviceOnce shared;
  std::vector<std::thread> th;
  std::vector<int> st(8, -1);
  for (int t = 0; t < 8; ++t)
    th.emplace_back([&, t] {
      st[t] = shared.run([](int* d) { *d = 2; return 0; }, [] { return 0; });
    });
  for (auto& x : th) x.join();
  for (int v : st)
    if (v != 0) return fail("concurrent status");
  int later = 0;
  shared.run([](int* d) { *d = 2; return 0; }, [&] { ++later; return 0; });
  if (later != 0) return fail("concurrent set-up not remembered");

  std::printf("ok\n");
  return 0;
}
