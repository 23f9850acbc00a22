// Shared definitions of the BM-Global CUDA library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string>
#include <vector>

#include "../../include/bm.h"

namespace bm {

// ----------------------------------------------------------------------------
// Error handling: every CUDA call is checked; failures become a bm_status and
// a message stored on the handle.  Nothing aborts or throws across the C ABI.
// ----------------------------------------------------------------------------
struct Error {
  bm_status code;
  std::string msg;
};

// A failed call throws; the runtime's last-error state is cleared first so
// that a later launch check does not report this failure again.
#define BM_CUDA(call)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      (void)cudaGetLastError();                                                         \
      throw ::bm::Error{e_ == cudaErrorMemoryAllocation ? BM_ERR_OOM : BM_ERR_CUDA,     \
                        std::string(#call) + ": " + cudaGetErrorString(e_)};            \
    }                                                                                   \
  } while (0)

#define BM_CHECK_LAUNCH() BM_CUDA(cudaGetLastError())

#define BM_REQUIRE(cond, code, text)                       \
  do {                                                     \
    if (!(cond)) throw ::bm::Error{(code), (text)};        \
  } while (0)

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int round_up4(int k) { return (k + 3) & ~3; }

// Device buffer owned by a handle (freed in the destructor).
template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  void alloc(size_t count) {
    if (count <= n && p) return;
    release();
    if (count == 0) count = 1;
    BM_CUDA(cudaMalloc(&p, count * sizeof(T)));
    n = count;
  }
  T* get() const { return p; }
};

// Number of SMs of the current device (cached).
int num_sms();

// True if ptr is a device (or managed) address.
bool is_device_ptr(const void* ptr);

// Raise `kernel`'s dynamic shared-memory limit to the device's opt-in
// maximum, once per process and device.  The limit is a per-function
// attribute shared by all host threads: setting it to each launch's own size
// right before the launch races with other threads' launches of the same
// kernel (a smaller value set in between makes their launch fail).
void allow_max_smem(const void* kernel);

}  // namespace bm
