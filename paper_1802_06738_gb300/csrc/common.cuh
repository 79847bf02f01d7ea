// Shared helpers of the pnoeom library: error plumbing, device buffers,
// the device context (stream + cuSOLVER handle).
#pragma once
#include <cuda_runtime.h>
#include <mutex>
#include <cusolverDn.h>
#include <cstdio>
#include <cstdint>
#include <string>
#include <vector>
#include <stdexcept>
#include "../../include/pnoeom.h"

namespace pnoeom {

// Library-internal exception carrying a pnoeom error code; the C entry points
// translate it into a return code and a thread-local message.
struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define PN_CUDA(call)                                                              \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      throw ::pnoeom::Error(e_ == cudaErrorMemoryAllocation ? PNOEOM_ERR_NOMEM      \
                                                            : PNOEOM_ERR_CUDA,     \
                            std::string(#call) + ": " + cudaGetErrorString(e_));   \
  } while (0)

#define PN_SOLVER(call)                                                            \
  do {                                                                             \
    cusolverStatus_t s_ = (call);                                                  \
    if (s_ != CUSOLVER_STATUS_SUCCESS)                                             \
      throw ::pnoeom::Error(PNOEOM_ERR_CUDA,                                       \
                            std::string(#call) + ": cusolver status " + std::to_string((int)s_)); \
  } while (0)

#define PN_CHECK(cond, code, msg)                                                  \
  do { if (!(cond)) throw ::pnoeom::Error((code), (msg)); } while (0)

// Per-host-thread caching device allocator.  Freed blocks are kept and reused
// by later allocations of the same thread; every thread of the library keeps to
// one stream for its device work, so a reused block is stream-ordered after the
// work that used it before.  trim() frees the calling thread's cached blocks; the caller must first
// synchronise the stream its device work runs on.  Allocation and trimming
// never overlap a CUDA-graph capture of another thread (capture_mutex).
void* pool_get(size_t bytes);
void pool_put(void* p, size_t bytes);
void pool_trim();
std::recursive_mutex& capture_mutex();
// Fault injection: after `after` further successful requests (0: the next one), one
// pool_get fails with PNOEOM_ERR_NOMEM; a negative value disables it.  live_alloc_bytes:
// bytes of blocks handed out by pool_get and not yet returned, over all threads.
void inject_alloc_failure(long long after);
long long live_alloc_bytes();

// Owning device buffer (cached allocator, see pool_get).  Counts bytes into a shared
// footprint counter so handles can report their device footprint.
template <typename T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  size_t* counter = nullptr;
  DBuf() = default;
  explicit DBuf(size_t count, size_t* ctr = nullptr) { alloc(count, ctr); }
  void alloc(size_t count, size_t* ctr = nullptr) {
    release();
    if (count) p = (T*)pool_get(count * sizeof(T));   // may throw: nothing recorded yet
    n = count;
    counter = ctr;
    if (counter) *counter += count * sizeof(T);
  }
  void release() {
    if (p) pool_put(p, n * sizeof(T));
    if (counter) *counter -= n * sizeof(T);
    p = nullptr; n = 0; counter = nullptr;
  }
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept { p = o.p; n = o.n; counter = o.counter; o.p = nullptr; o.n = 0; o.counter = nullptr; }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) { release(); p = o.p; n = o.n; counter = o.counter; o.p = nullptr; o.n = 0; o.counter = nullptr; }
    return *this;
  }
  ~DBuf() { release(); }
  T* get() const { return p; }
  void zero(cudaStream_t s) { if (n) PN_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), s)); }
  void upload(const T* h, size_t count, cudaStream_t s) {
    if (count) PN_CUDA(cudaMemcpyAsync(p, h, count * sizeof(T), cudaMemcpyHostToDevice, s));
  }
  void download(T* h, size_t count, cudaStream_t s) const {
    if (count) PN_CUDA(cudaMemcpyAsync(h, p, count * sizeof(T), cudaMemcpyDeviceToHost, s));
  }
};

// Makes `device` current for the scope of one C entry point and restores the
// caller's current device on the way out (also when an error is thrown), so a
// call never leaves another device current for the caller's later work.
struct DeviceScope {
  int prev = -1;
  explicit DeviceScope(int device) {
    PN_CUDA(cudaGetDevice(&prev));
    if (prev != device) PN_CUDA(cudaSetDevice(device));
  }
  ~DeviceScope() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
  DeviceScope(const DeviceScope&) = delete;
  DeviceScope& operator=(const DeviceScope&) = delete;
};

// Stage timer for tracing: when the environment variable PNOEOM_LOG_TIMING is
// set, mark() synchronises the stream and prints the seconds since the last mark.
struct StageTimer {
  cudaStream_t s;
  bool on;
  double t0;
  explicit StageTimer(cudaStream_t st);
  void mark(const char* what);
};

}  // namespace pnoeom

struct pnoeom_ctx {
  int device = 0;
  size_t budget = 0;
  cusolverDnHandle_t solver = nullptr;
};
