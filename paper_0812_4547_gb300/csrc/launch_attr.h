// launch_attr.h -- kernel attributes set once per device.
//
// A kernel's attributes (the dynamic shared memory it may ask for, its
// preferred shared-memory carveout) belong to each device's context, so a
// process that drives several devices must set them on every device it
// launches on.  These helpers remember, per device, what was set.
#pragma once

#include <cuda_runtime.h>

#include <mutex>

namespace rnnls {

constexpr int kAttrDevices = 64;  // devices remembered; higher ordinals set on every call

// Runs `set` the first time it is reached on the current device; later calls
// on that device return cudaSuccess without running it (a failed `set` is
// retried on the next call).
struct once_per_device {
  std::mutex m;
  bool done[kAttrDevices] = {};

  template <typename F>
  cudaError_t run(F &&set) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= kAttrDevices) return set();
    std::lock_guard<std::mutex> g(m);
    bool &d = done[dev];
    if (d) return cudaSuccess;
    e = set();
    if (e == cudaSuccess) d = true;
    return e;
  }
};

// The largest dynamic shared memory `func` was allowed on each device; grows
// it on the current device when a launch needs more.
struct smem_attr {
  std::mutex m;
  int bytes[kAttrDevices] = {};

  cudaError_t ensure(const void *func, size_t need) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= kAttrDevices) return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
    std::lock_guard<std::mutex> g(m);
    int &have = bytes[dev];
    if ((int)need <= have) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
    if (e == cudaSuccess) have = (int)need;
    return e;
  }
};

}  // namespace rnnls
