// Shared host-side utilities: error handling, device buffers, budget tracking.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <stdexcept>
#include <string>
#include <vector>

namespace mfns {

enum Status : int {
  kOk = 0, kErrArg = -1, kErrOom = -2, kErrBudget = -3, kErrUnsupported = -4,
  kErrCuda = -5, kErrTimeout = -6, kErrNotConverged = -7
};

struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#ifdef __FILE_NAME__
#define MFNS_SRC_FILE __FILE_NAME__
#else
#define MFNS_SRC_FILE __FILE__
#endif
#define MFNS_CUDA(expr)                                                                                   \
  do {                                                                                                    \
    cudaError_t e_ = (expr);                                                                              \
    if (e_ != cudaSuccess)                                                                                \
      throw ::mfns::Error(::mfns::kErrCuda, std::string(MFNS_SRC_FILE ":") + std::to_string(__LINE__) + \
                                                " " #expr ": " + cudaGetErrorString(e_));                 \
  } while (0)

// Per-context HBM accounting: every library allocation is charged against the budget
// (thread-safe: problems of one context may be created and destroyed from several threads).
struct Budget {
  size_t limit = 0, used = 0, peak = 0;
  std::mutex mu;
  void charge(size_t b) {
    std::lock_guard<std::mutex> lock(mu);
    if (limit && used + b > limit) throw Error(kErrBudget, "HBM budget exceeded");
    used += b;
    if (used > peak) peak = used;
  }
  void release(size_t b) {
    std::lock_guard<std::mutex> lock(mu);
    used -= b;
  }
};

class DevBuf {
 public:
  DevBuf() = default;
  DevBuf(Budget* bud, size_t bytes) { alloc(bud, bytes); }
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept { swap(o); }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) { free(); swap(o); }
    return *this;
  }
  ~DevBuf() { free(); }
  void alloc(Budget* bud, size_t bytes) {
    free();
    if (bytes == 0) return;
    if (bud) bud->charge(bytes);
    cudaError_t e = cudaMalloc(&p_, bytes);
    if (e != cudaSuccess) {
      if (bud) bud->release(bytes);
      p_ = nullptr;
      throw Error(kErrOom, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    bytes_ = bytes;
    bud_ = bud;
  }
  void free() {
    if (p_) {
      cudaFree(p_);
      if (bud_) bud_->release(bytes_);
    }
    p_ = nullptr;
    bytes_ = 0;
    bud_ = nullptr;
  }
  template <typename T> T* as() const { return reinterpret_cast<T*>(p_); }
  void* get() const { return p_; }
  size_t bytes() const { return bytes_; }

 private:
  void swap(DevBuf& o) {
    std::swap(p_, o.p_);
    std::swap(bytes_, o.bytes_);
    std::swap(bud_, o.bud_);
  }
  void* p_ = nullptr;
  size_t bytes_ = 0;
  Budget* bud_ = nullptr;
};

template <typename T>
DevBuf upload(Budget* bud, const std::vector<T>& v) {
  DevBuf b(bud, v.size() * sizeof(T));
  if (!v.empty()) MFNS_CUDA(cudaMemcpy(b.get(), v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return b;
}

inline size_t esize(int prec) { return prec == 0 ? 8 : 4; }  // 0 = fp64, 1 = fp32

}  // namespace mfns
