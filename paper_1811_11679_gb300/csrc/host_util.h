// host_util.h -- host-side helpers shared by the library's host units: CUDA
// error and failure exceptions (caught at the C ABI and turned into a
// hande_status) and device allocation through the context's allocator.
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "engine.h"

namespace hande {

struct CudaError {
  cudaError_t e;
  const char* what;
};

#define CK(call)                                      \
  do {                                                \
    cudaError_t _e = (call);                          \
    if (_e != cudaSuccess) throw CudaError{_e, #call}; \
  } while (0)

struct Fail {
  hande_status code;
  std::string msg;
};

// device memory of the context (its allocator, else cudaMalloc), freed with it
inline void* dev_alloc(Engine& E, size_t bytes) {
  bytes = (bytes + 255) & ~size_t(255);
  if (bytes == 0) bytes = 256;
  void* p = nullptr;
  if (E.has_alloc) {
    p = E.alloc.alloc(bytes, E.alloc.user);
    if (!p) throw Fail{HANDE_ERR_NOMEM, "device allocation failed (" + std::to_string(bytes) + " bytes)"};
  } else {
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      throw Fail{HANDE_ERR_NOMEM, "cudaMalloc failed (" + std::to_string(bytes) + " bytes)"};
    }
  }
  E.blocks.push_back({p, bytes});
  return p;
}
template <typename T>
T* dalloc(Engine& E, size_t count) {
  return static_cast<T*>(dev_alloc(E, count * sizeof(T)));
}

}  // namespace hande
