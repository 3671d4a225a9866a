"""The library's per-device launch caches (kernel attribute opt-ins,
occupancies, symbol addresses, SM counts) key on the current device.  The
cache template is compiled on the host with g++ against a fake
cudaGetDevice, so no GPU is needed: a value stored while device 0 is current
is not seen on device 1, each device keeps its own value, and a device index
that cannot be cached yields no slot."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2407_02100_gb300", "csrc")

PROG = r'''
#include "per_device.h"
#include <cstdio>

static int g_fake_device = 0;
static cudaError_t g_fake_status = cudaSuccess;
extern "C" cudaError_t cudaGetDevice(int* d) { *d = g_fake_device; return g_fake_status; }

int main() {
  gmg::PerDevice<int> cache;
  g_fake_device = 0;
  int* a = cache.get();
  if (!a || *a != 0) return 1;
  *a = 5;
  g_fake_device = 1;
  int* b = cache.get();
  if (!b || b == a || *b != 0) return 2;   // device 1 starts empty
  *b = 7;
  g_fake_device = 0;
  if (cache.get() != a || *cache.get() != 5) return 3;
  g_fake_device = 1;
  if (*cache.get() != 7) return 4;
  g_fake_device = gmg::kMaxDevices;          // beyond the table
  if (cache.get() != nullptr) return 5;
  g_fake_device = -1;
  if (cache.get() != nullptr) return 6;
  g_fake_device = 0;
  g_fake_status = cudaErrorNoDevice;         // cudaGetDevice fails
  if (cache.get() != nullptr || gmg::current_device() != -1) return 7;
  std::puts("ok");
  return 0;
}
'''


def test_per_device_cache_keys_on_the_current_device(tmp_path):
    gxx = shutil.which("g++")
    inc = "/usr/local/cuda/include"
    if not gxx or not os.path.exists(os.path.join(inc, "cuda_runtime_api.h")):
        pytest.skip("needs g++ and the CUDA headers")
    src = tmp_path / "per_device_test.cpp"
    exe = tmp_path / "per_device_test"
    src.write_text(PROG)
    subprocess.run([gxx, "-std=c++17", "-O1", f"-I{CSRC}", f"-I{inc}", str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    res = subprocess.run([str(exe)], capture_output=True, text=True)
    assert res.returncode == 0 and res.stdout.strip() == "ok", (res.returncode, res.stdout, res.stderr)
