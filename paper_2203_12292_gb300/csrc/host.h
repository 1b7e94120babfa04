// Host-side helpers of libgcmg's C ABI: error propagation (no exception
// crosses the ABI), checked CUDA calls and owning device buffers.
#pragma once

#include <cuda_runtime.h>

#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "gcmg.h"

namespace gcmg {

// message of the last failed call of this host thread
inline thread_local std::string g_err;

struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

inline void ck(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error(e == cudaErrorMemoryAllocation ? GCMG_ERR_OOM : GCMG_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
  }
}

// first failed kernel launch (or launch-attribute call) of this host thread
// that no check has reported yet; the launch helpers record it, every entry
// point reports it
inline thread_local cudaError_t g_launch_err = cudaSuccess;
inline void note_launch_error(cudaError_t e) {
  if (e != cudaSuccess && g_launch_err == cudaSuccess) g_launch_err = e;
}
// throw for a recorded launch failure or a pending CUDA error of this thread
inline void ck_launches(const char* what) {
  const cudaError_t e = g_launch_err;
  g_launch_err = cudaSuccess;
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error(GCMG_ERR_CUDA, std::string(what) + ": kernel launch failed: " + cudaGetErrorString(e));
  }
  ck(cudaGetLastError(), what);
}

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  void alloc(size_t n) {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = n;
    if (n) ck(cudaMalloc(&p, n), "cudaMalloc");
  }
  template <typename T>
  void upload(const std::vector<T>& v, cudaStream_t s) {
    alloc(v.size() * sizeof(T));
    if (!v.empty()) ck(cudaMemcpyAsync(p, v.data(), bytes, cudaMemcpyHostToDevice, s), "upload");
  }
  template <typename T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

// run f, turn exceptions into GCMG_ERR_* codes and the thread's message
template <typename F>
int guarded(F&& f) {
  g_launch_err = cudaSuccess;
  try {
    f();
    if (g_launch_err != cudaSuccess) ck_launches("launch");
    return GCMG_OK;
  } catch (const Error& e) {
    g_err = e.what();
    return e.code;
  } catch (const std::bad_alloc&) {
    g_err = "host allocation failed";
    return GCMG_ERR_OOM;
  } catch (const std::exception& e) {
    g_err = e.what();
    return GCMG_ERR_INTERNAL;
  }
}

}  // namespace gcmg
