// Host-side checks of caller pointers and of the calling thread's current
// device.  Library plumbing; the paper has no counterpart.
#pragma once

#include <cuda_runtime.h>

namespace snaps {

// Where a caller's buffer lives, as the library may use it on `device`.
enum class PtrKind {
    Host,     // host memory (pageable or pinned): reached through copies
    Device,   // memory the kernels on `device` may read and write directly
    Foreign,  // device memory of another GPU: its kernels would fault there
};

// The decision from cudaPointerGetAttributes' answer (type and owning
// device).  Managed memory migrates on demand, so every device may use it.
inline PtrKind ptr_kind_of(cudaMemoryType type, int owner, int device)
{
    if (type == cudaMemoryTypeManaged) return PtrKind::Device;
    if (type == cudaMemoryTypeDevice) return owner == device ? PtrKind::Device : PtrKind::Foreign;
    return PtrKind::Host;
}

inline PtrKind ptr_kind(const void *p, int device)
{
    cudaPointerAttributes a;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // an unregistered host pointer is not an error
        return PtrKind::Host;
    }
    return ptr_kind_of(a.type, a.device, device);
}

// Makes `device` current for the lifetime of the object and restores the
// calling thread's previous device afterwards, on every return path.
class DeviceScope {
  public:
    explicit DeviceScope(int device)
    {
        if (cudaGetDevice(&prev_) != cudaSuccess) {
            cudaGetLastError();
            prev_ = -1;
        }
        err_ = prev_ == device ? cudaSuccess : cudaSetDevice(device);
    }
    ~DeviceScope()
    {
        if (prev_ >= 0 && err_ == cudaSuccess) cudaSetDevice(prev_);
    }
    cudaError_t error() const { return err_; }
    DeviceScope(const DeviceScope &) = delete;
    DeviceScope &operator=(const DeviceScope &) = delete;

  private:
    int prev_ = -1;
    cudaError_t err_ = cudaSuccess;
};

}  // namespace snaps
