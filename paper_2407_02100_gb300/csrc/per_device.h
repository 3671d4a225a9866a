// Per-device caches of launch set-up.  The CUDA runtime keeps a kernel's
// dynamic shared-memory opt-in, and the addresses of __device__ symbols, per
// device; occupancy and the SM count are properties of the device.  Host code
// that caches any of them keeps one slot per device index, so that a process
// driving several GPUs sets each kernel up on each device and passes every
// kernel the symbol addresses of the device it runs on.
#pragma once
#include <cuda_runtime_api.h>

namespace gmg {

constexpr int kMaxDevices = 64;

// Index of the current device, or -1 if it cannot be read or is >= kMaxDevices.
inline int current_device() {
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices) return -1;
  return d;
}

// One value per device, zero-initialised; get() returns the current device's
// slot, or nullptr when current_device() fails.  Not synchronised: a slot is
// written by the first launch on its device, with the same value by every
// writer.
template <typename V>
struct PerDevice {
  V slot[kMaxDevices] = {};
  V* get() {
    const int d = current_device();
    return d < 0 ? nullptr : &slot[d];
  }
};

}  // namespace gmg
