"""The once-per-device flag the propagation launchers use to opt each kernel
in to its shared memory (csrc/per_device.h).

A kernel's dynamic shared-memory limit is an attribute of the kernel on one
device, so the launchers must set it on every device they launch on, not
once per process, and must not record success when the call failed.  The
helper has no CUDA dependency, so this test compiles a small C++ driver with
the host compiler and checks the logic on the CPU (a run on two real devices
is not possible where each test run gets one GPU).
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2203_06117_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <thread>
#include <vector>
#include "per_device.h"

static int calls[80];
static int fail_left[80];

int action(int dev) {
  ++calls[dev];
  if (fail_left[dev] > 0) { --fail_left[dev]; return 7; }
  return 0;
}

int main() {
  int bad = 0;
  auto check = [&](bool ok, const char* what) { if (!ok) { std::printf("FAIL %s\n", what); ++bad; } };
  gatspi_host::PerDeviceOnce once;
  // first use on device 0 runs the action and sets the flag; later uses do not run it
  check(once.run(0, [] { return action(0); }) == 0, "device 0 first call succeeds");
  check(once.run(0, [] { return action(0); }) == 0, "device 0 second call succeeds");
  check(calls[0] == 1, "device 0 action ran once");
  check(once.done(0), "device 0 flag set");
  // another device is independent: its flag is clear until its own action ran
  check(!once.done(1), "device 1 flag clear");
  check(once.run(1, [] { return action(1); }) == 0 && calls[1] == 1 && once.done(1), "device 1 set on its own");
  // a failure is returned, leaves the flag clear, and the next call retries
  fail_left[2] = 2;
  check(once.run(2, [] { return action(2); }) == 7, "failure returned");
  check(!once.done(2), "failure leaves flag clear");
  check(once.run(2, [] { return action(2); }) == 7, "second failure returned");
  check(once.run(2, [] { return action(2); }) == 0 && once.done(2) && calls[2] == 3, "retry after failure");
  check(once.run(2, [] { return action(2); }) == 0 && calls[2] == 3, "no call after success");
  // devices beyond the table get no flag: the action runs every time
  check(once.run(70, [] { return action(70); }) == 0 && once.run(70, [] { return action(70); }) == 0,
        "untracked device succeeds");
  check(calls[70] == 2 && !once.done(70), "untracked device runs every call");
  check(once.run(-1, [] { return 0; }) == 0 && !once.done(-1), "negative device untracked");
  // many threads at once on a fresh device: all succeed, the flag ends set
  gatspi_host::PerDeviceOnce shared;
  std::vector<std::thread> ts;
  std::vector<int> rc(16, -1);
  for (int k = 0; k < 16; ++k)
    ts.emplace_back([&, k] { rc[k] = shared.run(5, [] { return 0; }); });
  for (auto& t : ts) t.join();
  bool all_ok = true;
  for (int r : rc) all_ok = all_ok && r == 0;
  check(all_ok && shared.done(5), "concurrent first use");
  std::printf(bad ? "FAILED\n" : "OK\n");
  return bad ? 1 : 0;
}
"""


def test_per_device_once(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "drv.cpp"
    src.write_text(DRIVER)
    exe = tmp_path / "drv"
    subprocess.check_call([cxx, "-std=c++17", "-O1", "-pthread", "-I" + CSRC, str(src), "-o", str(exe)])
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip().endswith("OK"), out.stdout + out.stderr
