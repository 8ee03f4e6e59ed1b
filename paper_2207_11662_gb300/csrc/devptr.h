// Which pointers a kernel launched on the current device may read directly.
//
// Plain C++ over the CUDA runtime's pointer-attribute struct (no device code, no
// runtime calls), so the rule can be checked on a machine without a GPU.
#pragma once

#include <cuda_runtime_api.h>

namespace homln {

// True when memory with attributes `at` can be read by a kernel running on
// `current_device` without peer access: managed memory, or device memory that
// lives on that same device. Host, registered-host and unregistered memory, and
// device memory of another GPU, are refused (reading another GPU's memory
// through the unified address space faults when peer access is off).
inline bool device_pointer_usable(const cudaPointerAttributes &at, int current_device) {
    if (at.type == cudaMemoryTypeManaged) return true;
    return at.type == cudaMemoryTypeDevice && at.device == current_device;
}

}  // namespace homln
