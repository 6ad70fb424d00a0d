"""Per-device launch set-up (csrc/device_cache.h) on the host: a C++ driver
built with g++ runs many threads over several fake device ordinals and checks
that the set-up runs exactly once per device, that every caller sees that
device's value, that a failed set-up stores nothing (the next call retries) and
that out-of-range ordinals are refused. No GPU is involved: the class holds no
CUDA types."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2508_03065_gb300", "csrc")

DRIVER = r"""
#include <atomic>
#include <cstdio>
#include <thread>
#include <vector>
#include "device_cache.h"

int main() {
  msrc::PerDevice cache;
  constexpr int kDev = 6, kThreads = 16, kCalls = 2000;
  std::atomic<int> inits[kDev] = {};
  std::atomic<int> bad{0};
  std::vector<std::thread> pool;
  for (int t = 0; t < kThreads; ++t)
    pool.emplace_back([&, t] {
      for (int i = 0; i < kCalls; ++i) {
        const int dev = (t + i) % kDev;
        int v = 0;
        const int st = cache.get(dev, [&](int* out) {
          inits[dev].fetch_add(1);
          std::this_thread::yield();
          *out = 100 + dev;
          return 0;
        }, &v);
        if (st != 0 || v != 100 + dev) bad.fetch_add(1);
      }
    });
  for (auto& th : pool) th.join();
  for (int d = 0; d < kDev; ++d)
    if (inits[d].load() != 1) { std::printf("device %d set up %d times\n", d, inits[d].load()); return 1; }
  if (bad.load()) { std::printf("%d wrong values\n", bad.load()); return 2; }
  // a failed set-up stores nothing; the next call runs it again
  msrc::PerDevice c2;
  int v = 0, runs = 0;
  if (c2.get(3, [&](int* out) { ++runs; return 7; }, &v) != 7) return 3;
  if (c2.get(3, [&](int* out) { ++runs; *out = 5; return 0; }, &v) != 0 || v != 5 || runs != 2) return 4;
  if (c2.get(3, [&](int* out) { ++runs; *out = 9; return 0; }, &v) != 0 || v != 5 || runs != 2) return 5;
  // a set-up that reports success without a value is an error, not a stored 0
  if (c2.get(4, [&](int* out) { *out = 0; return 0; }, &v) != -2) return 6;
  // ordinals outside the table are refused
  if (c2.get(-1, [&](int* out) { *out = 1; return 0; }, &v) != -1) return 7;
  if (c2.get(msrc::kMaxDevices, [&](int* out) { *out = 1; return 0; }, &v) != -1) return 8;
  std::printf("ok\n");
  return 0;
}
"""


def test_per_device_setup_runs_once_per_device(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    src = tmp_path / "driver.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "driver"
    r = subprocess.run([gxx, "-std=c++17", "-O1", "-pthread", "-I", CSRC, str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip() == "ok"
