// Host staging memory of the serving queue: an arena of large page-locked
// chunks carved by a first-fit free list with coalescing.
//
// A request's inputs are copied into staging when it is submitted, and its
// outputs land there when it retires.  Page-locked memory is what lets the
// copies to and from the device run asynchronously at full link speed, but
// allocating it (cudaMallocHost) takes milliseconds per call and grows with
// the size.  The arena allocates chunks of at least kChunkBytes and reuses
// the space of retired requests for any later request, whatever its shape.
// Chunks are kept until the arena is destroyed.  With `pinned` false the
// chunks come from malloc (the queue's fake-device mode), so the same
// allocator logic runs without a GPU.
//
// Large copies into staging are split across threads (parallel_copy): one
// core copies well below the host memory bandwidth.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <iterator>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

namespace sense {

class PinnedArena {
 public:
  static constexpr size_t kAlign = 256;
  static constexpr size_t kChunkBytes = (size_t)256 << 20;

  explicit PinnedArena(bool pinned) : pinned_(pinned) {}
  ~PinnedArena() {
    for (Chunk& c : chunks_) release(c.base);
  }
  PinnedArena(const PinnedArena&) = delete;
  PinnedArena& operator=(const PinnedArena&) = delete;

  // At least `bytes` of staging, kAlign-aligned; nullptr if the host is out
  // of (page-locked) memory.
  void* get(size_t bytes) {
    const size_t need = round(std::max<size_t>(bytes, 1));
    {
      std::lock_guard<std::mutex> lock(mu_);
      if (void* p = take(need)) return p;
    }
    // new chunk, allocated outside the lock (cudaMallocHost is slow); chunks
    // grow with what is already reserved, so a growing load pays for few
    size_t size;
    {
      std::lock_guard<std::mutex> lock(mu_);
      size = std::max(std::max(kChunkBytes, need), round(reserved_ / 2));
    }
    char* base = static_cast<char*>(acquire(size));
    if (!base) return nullptr;
    std::lock_guard<std::mutex> lock(mu_);
    Chunk c;
    c.base = base;
    c.size = size;
    c.free[0] = size;
    chunks_.push_back(std::move(c));
    reserved_ += size;
    return take(need);  // fits: the new chunk is free and large enough
  }

  // One chunk of `bytes` up front (queue creation), so the first requests
  // do not pay for page-locking.  Returns false if the host refused it.
  bool reserve(size_t bytes) {
    if (bytes == 0) return true;
    const size_t size = round(bytes);
    char* base = static_cast<char*>(acquire(size));
    if (!base) return false;
    std::lock_guard<std::mutex> lock(mu_);
    Chunk c;
    c.base = base;
    c.size = size;
    c.free[0] = size;
    chunks_.push_back(std::move(c));
    reserved_ += size;
    return true;
  }

  void put(void* p) {
    if (!p) return;
    std::lock_guard<std::mutex> lock(mu_);
    auto it = live_.find(p);
    if (it == live_.end()) return;
    const Block b = it->second;
    live_.erase(it);
    in_use_ -= b.len;
    auto& fl = chunks_[b.chunk].free;
    size_t off = b.off, len = b.len;
    auto next = fl.lower_bound(off);
    if (next != fl.end() && next->first == off + len) {  // merge with the following free block
      len += next->second;
      next = fl.erase(next);
    }
    if (next != fl.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {  // merge with the preceding free block
        prev->second += len;
        return;
      }
    }
    fl[off] = len;
  }

  size_t reserved() {
    std::lock_guard<std::mutex> lock(mu_);
    return reserved_;
  }
  size_t in_use() {
    std::lock_guard<std::mutex> lock(mu_);
    return in_use_;
  }
  size_t chunks() {
    std::lock_guard<std::mutex> lock(mu_);
    return chunks_.size();
  }

 private:
  struct Chunk {
    char* base = nullptr;
    size_t size = 0;
    std::map<size_t, size_t> free;  // offset -> length, disjoint and not adjacent
  };
  struct Block {
    size_t chunk, off, len;
  };

  static size_t round(size_t b) { return (b + kAlign - 1) & ~(kAlign - 1); }

  // First fit over the chunks in creation order; caller holds mu_.
  void* take(size_t need) {
    for (size_t ci = 0; ci < chunks_.size(); ++ci) {
      auto& fl = chunks_[ci].free;
      for (auto it = fl.begin(); it != fl.end(); ++it) {
        if (it->second < need) continue;
        const size_t off = it->first, rest = it->second - need;
        fl.erase(it);
        if (rest) fl[off + need] = rest;
        void* p = chunks_[ci].base + off;
        live_[p] = Block{ci, off, need};
        in_use_ += need;
        return p;
      }
    }
    return nullptr;
  }

  void* acquire(size_t size) {
    if (!pinned_) return std::malloc(size);
    void* p = nullptr;
    return cudaMallocHost(&p, size) == cudaSuccess ? p : nullptr;
  }
  void release(void* p) {
    if (!pinned_)
      std::free(p);
    else
      cudaFreeHost(p);
  }

  const bool pinned_;
  std::mutex mu_;
  std::vector<Chunk> chunks_;
  std::unordered_map<void*, Block> live_;
  size_t reserved_ = 0, in_use_ = 0;
};

// memcpy, split over up to 8 threads (pieces of at least 2 MiB) for copies
// of 4 MiB and more.
inline void parallel_copy(void* dst, const void* src, size_t bytes) {
  constexpr size_t kPiece = (size_t)2 << 20;
  const size_t hw = std::max(1u, std::thread::hardware_concurrency());
  const size_t parts = std::min<size_t>(std::min<size_t>(8, hw), bytes / kPiece);
  if (parts < 2) {
    std::memcpy(dst, src, bytes);
    return;
  }
  const size_t step = ((bytes + parts - 1) / parts + 4095) & ~(size_t)4095;
  char* d = static_cast<char*>(dst);
  const char* s = static_cast<const char*>(src);
  std::vector<std::thread> workers;
  size_t done_to = step;  // bytes [0, done_to) are this thread's or a worker's
  for (size_t i = 1; i < parts; ++i) {
    const size_t off = i * step;
    if (off >= bytes) break;
    const size_t len = std::min(step, bytes - off);
    try {
      workers.emplace_back([=] { std::memcpy(d + off, s + off, len); });
    } catch (...) {  // no thread to be had: copy the rest here (no exception crosses the C ABI)
      break;
    }
    done_to = off + len;
  }
  std::memcpy(d, s, std::min(step, bytes));
  if (done_to < bytes) std::memcpy(d + done_to, s + done_to, bytes - done_to);
  for (std::thread& t : workers) t.join();
}

}  // namespace sense
