// dbbc_count_noalloc: counting for callers that must not allocate device
// memory. Some callers cannot call cudaMalloc (or any allocating routine)
// while they count: a serving loop that runs under a fixed device-memory
// budget owned by another framework's allocator, code that must not touch the
// device allocator while other streams are being captured into CUDA graphs,
// or embedded hosts that set up all memory at start-up. For them this entry
// point takes its scratch from one fixed array compiled into the library
// instead of allocating it per call.
//
// The scratch is a file-scope __device__ array of kNoAllocScratchBytes
// (32 MiB). Every GPU that loads the library holds it until the process
// exits. In host code the array's name is only a host-side stand-in, so its
// device address is taken with cudaGetSymbolAddress, once per device, the
// first time this entry point runs with that device current.
#include <mutex>
#include <vector>

#include "internal.h"
#include "common.cuh"

namespace dbbc {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
constexpr size_t kNoAllocHeaderBytes = 256;  // status word and work-item counter

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch on the current device (set up once per
// device; cudaGetSymbolAddress allocates nothing).
static unsigned char* noalloc_scratch_address() {
  static std::mutex mu;
  static std::vector<void*> addr;
  int dev = 0;
  DBBC_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  if ((int)addr.size() <= dev) addr.resize((size_t)dev + 1, nullptr);
  if (!addr[(size_t)dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      (void)cudaGetLastError();
      throw Error{DBBC_ECUDA, "cudaGetSymbolAddress(g_noalloc_scratch)"};
    }
    addr[(size_t)dev] = p;
  }
  return static_cast<unsigned char*>(addr[(size_t)dev]);
}

}  // namespace dbbc

using namespace dbbc;

extern "C" dbbc_status dbbc_count_noalloc(const dbbc_graph* g, void* cuda_stream, uint64_t* d_out) {
  if (!g || !d_out) return DBBC_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  try {
    unsigned char* base = noalloc_scratch_address();
    unsigned* d_status = reinterpret_cast<unsigned*>(base);
    int* d_next = reinterpret_cast<int*>(base + 64);
    uint32_t* cursors = reinterpret_cast<uint32_t*>(base + kNoAllocHeaderBytes);
    enqueue_count_prealloc(g, s, reinterpret_cast<unsigned long long*>(d_out), d_status, d_next, cursors,
                           kNoAllocScratchBytes - kNoAllocHeaderBytes);
    return DBBC_OK;
  } catch (const Error& e) {
    return e.status;
  } catch (...) {
    return DBBC_EINTERNAL;
  }
}
