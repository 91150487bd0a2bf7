// Shared device/host helpers for the dbbc CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <new>
#include <stdexcept>
#include <vector>

#include "../../include/dbbc.h"

namespace dbbc {

constexpr uint32_t kEmptyKey = 0xFFFFFFFFu;
constexpr unsigned kFullMask = 0xFFFFFFFFu;
constexpr int kNumSMs = 152;  // GB300: 2 dies x 76 SMs (used only as a default)

// Status raised inside the library and turned into a dbbc_status at the ABI.
struct Error {
  dbbc_status status;
  const char* where;
};

#define DBBC_CUDA(call)                                           \
  do {                                                            \
    cudaError_t e_ = (call);                                      \
    if (e_ != cudaSuccess) {                                      \
      (void)cudaGetLastError();                                   \
      throw ::dbbc::Error{e_ == cudaErrorMemoryAllocation ? DBBC_ENOMEM : DBBC_ECUDA, #call}; \
    }                                                             \
  } while (0)

void note_launch();                // counts kernels launched by the library
void note_launches(uint64_t k);    // k kernels launched at once (a CUDA graph replay)
uint64_t launches_so_far();
#define DBBC_LAUNCH_CHECK()          \
  do {                               \
    ::dbbc::note_launch();           \
    DBBC_CUDA(cudaGetLastError());   \
  } while (0)

inline int bits_for(uint64_t x) {  // bits needed to represent values in [0, x]
  int b = 0;
  while (b < 64 && (x >> b) != 0) b++;
  return b;
}

template <typename T>
inline T ceil_div(T a, T b) {
  return (a + b - 1) / b;
}

// ---------------------------------------------------------------- allocator
void* dev_alloc(size_t bytes, cudaStream_t s);
void dev_free(void* p, cudaStream_t s);

// Scratch allocations released (stream-ordered) when the scope ends.
class Scratch {
 public:
  explicit Scratch(cudaStream_t s) : s_(s) {}
  ~Scratch() {
    for (void* p : ptrs_) dev_free(p, s_);
  }
  template <typename T>
  T* get(size_t n) {
    if (n == 0) n = 1;
    void* p = dev_alloc(n * sizeof(T), s_);
    if (!p) throw Error{DBBC_ENOMEM, "Scratch::get"};
    ptrs_.push_back(p);
    return static_cast<T*>(p);
  }
  Scratch(const Scratch&) = delete;
  Scratch& operator=(const Scratch&) = delete;

 private:
  cudaStream_t s_;
  std::vector<void*> ptrs_;
};

// ---------------------------------------------------------------- device helpers
__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFullMask, x, o);
  return x;
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// Block-wide sum of two u64 values, then one global atomic pair per block.
// Every thread of the block must call it.
template <int THREADS>
__device__ __forceinline__ void block_add_pair(uint64_t a, uint64_t b, unsigned long long* out) {
  __shared__ unsigned long long red[2][THREADS / 32];
  a = warp_sum_u64(a);
  b = warp_sum_u64(b);
  const int w = threadIdx.x >> 5;
  if (lane_id() == 0) {
    red[0][w] = a;
    red[1][w] = b;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    uint64_t x = threadIdx.x < THREADS / 32 ? red[0][threadIdx.x] : 0;
    uint64_t y = threadIdx.x < THREADS / 32 ? red[1][threadIdx.x] : 0;
    x = warp_sum_u64(x);
    y = warp_sum_u64(y);
    if (threadIdx.x == 0) {
      if (x) atomicAdd(&out[0], (unsigned long long)x);
      if (y) atomicAdd(&out[1], (unsigned long long)y);
    }
  }
}

}  // namespace dbbc
