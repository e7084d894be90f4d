// Checks on caller-owned buffers that the library hands to its kernels or to
// device-side copies as they are (CHEM_MEM_DEVICE arguments and the
// allocation-free entry point).
#pragma once

#include <cuda_runtime.h>

#include <cstring>
#include <string>

namespace chemgpu {

// Empty if p is memory of device dev or managed memory, else why not: a
// kernel given a host pointer, or another device's memory without peer
// access, would fault.  cudaPointerGetAttributes allocates nothing; a failed
// query also sets the runtime's last error, which is reset here.
inline std::string device_buffer_problem(const void *p, int dev, const char *name) {
  cudaPointerAttributes a;
  std::memset(&a, 0, sizeof(a));
  const cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return std::string(name) + " is not a device pointer (" + cudaGetErrorString(e) + ")";
  }
  if (a.type == cudaMemoryTypeManaged) return std::string();
  if (a.type != cudaMemoryTypeDevice) return std::string(name) + " must be memory of the current device, not host memory";
  if (a.device != dev)
    return std::string(name) + " is memory of device " + std::to_string(a.device) + ", not of the current device " +
           std::to_string(dev);
  return std::string();
}

}  // namespace chemgpu
