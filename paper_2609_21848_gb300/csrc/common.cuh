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

// Status bits written by kernels (device status word).
enum : unsigned {
  DBBC_DEV_HASH_FULL = 1u,  // a shared hash table ran out of slots (tier sizing bug)
  DBBC_DEV_RANGE = 2u,      // an index left its array (checked builds only)
};

// ---------------------------------------------------------------- checked builds
// A library built with -DDBBC_CHECKED=1 tests the indexes its kernels derive
// from graph data before each access: CSR row and entry positions, the
// shared-memory address of every window counter, cursor and list slots, and
// per-vertex / per-edge output positions. A failed test skips the access and
// sets DBBC_DEV_RANGE in a flag word of the translation unit; the host
// collects every unit's word with checked_take_all(). In a regular build
// DBBC_CHECK(cond) is the constant true and generates no code.
#ifndef DBBC_CHECKED
#define DBBC_CHECKED 0
#endif

void checked_register(unsigned (*take)());
// OR of every unit's flag word since the last call, then cleared (synchronizes
// the current device); 0 without synchronizing in a regular build.
unsigned checked_take_all();

#if DBBC_CHECKED
static __device__ unsigned g_checked_flags;

__device__ __forceinline__ bool checked_ok(bool ok) {
  if (!ok) atomicOr(&g_checked_flags, DBBC_DEV_RANGE);
  return ok;
}
#define DBBC_CHECK(cond) (::dbbc::checked_ok(cond))

namespace {
// Registers this translation unit's flag word with the collector.
struct CheckedUnit {
  static unsigned take() {
    unsigned h = 0;
    const unsigned z = 0;
    if (cudaMemcpyFromSymbol(&h, g_checked_flags, sizeof(h)) != cudaSuccess) {
      (void)cudaGetLastError();
      return DBBC_DEV_RANGE;  // an unreadable flag word counts as a failed check
    }
    if (h && cudaMemcpyToSymbol(g_checked_flags, &z, sizeof(z)) != cudaSuccess) (void)cudaGetLastError();
    return h;
  }
  CheckedUnit() { checked_register(&take); }
};
static CheckedUnit checked_unit_;
}  // namespace
#else
#define DBBC_CHECK(cond) true
#endif

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
