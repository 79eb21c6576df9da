// Device scratch keyed by (device, stream).  Work queued on one stream
// reuses that stream's buffer in stream order; work on different streams,
// which may run at the same time (several k-points of pcx_solve in flight),
// never shares a buffer.  Streams are expected to be long-lived (a pool):
// a slot stays until the process exits.
#pragma once

#include <cuda_runtime.h>

#include <mutex>
#include <vector>

namespace pcx {

class StreamScratch {
 public:
  // a buffer of at least `bytes` for work on stream s of the current device
  cudaError_t get(cudaStream_t s, size_t bytes, void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu_);
    Slot* slot = nullptr;
    for (Slot& sl : slots_)
      if (sl.dev == dev && sl.s == s) slot = &sl;
    if (!slot) {
      slots_.push_back(Slot{dev, s, nullptr, 0});
      slot = &slots_.back();
    }
    if (bytes > slot->bytes) {
      if (slot->p) {
        // the old buffer may still be read by queued work
        if ((e = cudaDeviceSynchronize()) != cudaSuccess) return e;
        cudaFree(slot->p);
      }
      slot->p = nullptr;
      slot->bytes = 0;
      if ((e = cudaMalloc(&slot->p, bytes)) != cudaSuccess) return e;
      slot->bytes = bytes;
    }
    *out = slot->p;
    return cudaSuccess;
  }
  // free the buffer of stream s (call before destroying the stream)
  void release(cudaStream_t s) {
    std::lock_guard<std::mutex> lock(mu_);
    for (size_t i = 0; i < slots_.size(); ++i)
      if (slots_[i].s == s) {
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(slots_[i].dev);
        cudaStreamSynchronize(s);
        cudaFree(slots_[i].p);
        cudaSetDevice(cur);
        slots_.erase(slots_.begin() + (long)i);
        --i;
      }
  }
  // capacity of the stream's buffer (0 if none)
  size_t capacity(cudaStream_t s) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    std::lock_guard<std::mutex> lock(mu_);
    for (const Slot& sl : slots_)
      if (sl.dev == dev && sl.s == s) return sl.bytes;
    return 0;
  }

 private:
  struct Slot {
    int dev;
    cudaStream_t s;
    void* p;
    size_t bytes;
  };
  std::mutex mu_;
  std::vector<Slot> slots_;
};

}  // namespace pcx
