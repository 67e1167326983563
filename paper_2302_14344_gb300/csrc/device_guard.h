// DeviceGuard: every C-ABI call that touches a device makes the simulation's (or network's)
// device current for the call's duration and then restores the caller's current device, so a
// process that drives several GPUs keeps the device it selected.
#pragma once
#include <cuda_runtime.h>

namespace subadmm {

struct DeviceGuard {
    int prev = -1;                 // device to restore, -1 when nothing changed
    cudaError_t err = cudaSuccess; // result of making `dev` current
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) err = cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() { if (prev >= 0) cudaSetDevice(prev); }
    DeviceGuard(const DeviceGuard &) = delete;
    DeviceGuard &operator=(const DeviceGuard &) = delete;
};

}  // namespace subadmm
