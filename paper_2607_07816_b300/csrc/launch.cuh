// Programmatic dependent launch for the kernels of one gate or truncation.
//
// A kernel launched with launch_pdl may be scheduled onto the SMs while the
// kernel before it in the stream is still finishing, which hides the launch
// latency between the short kernels of a step.  Every such kernel starts
// with pdl_prologue(): griddepcontrol.wait blocks until the previous grid
// has completed and its writes are visible (so nothing the kernel reads can
// be stale), and griddepcontrol.launch_dependents lets the next kernel be
// scheduled in turn.  Both instructions do nothing when the kernel was
// launched without the attribute.
#pragma once

#include <cuda_runtime.h>

#include <mutex>
#include <utility>

namespace sv {

__device__ __forceinline__ void pdl_prologue() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... P, typename... A>
inline cudaError_t launch_pdl(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

// One-time host set-up per device.  A kernel's attributes (its dynamic
// shared-memory limit) belong to that kernel on one device, so they are set
// once for every device the library runs on: run(f) calls f the first time
// it is called with a given device current (thread-safe; concurrent callers
// wait for the first) and returns the error f returned there, on that call
// and on every later one with that device.
class DeviceOnce {
 public:
  static constexpr int kMaxDevices = 64;
  template <typename F>
  cudaError_t run(F&& f) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::call_once(flag_[dev], [&] { err_[dev] = f(); });
    return err_[dev];
  }

 private:
  std::once_flag flag_[kMaxDevices];
  cudaError_t err_[kMaxDevices] = {};
};

}  // namespace sv
