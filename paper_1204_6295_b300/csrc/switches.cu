// Test switches of the library (disc_set_test_switches in include/disc.h).
//
// The switches select alternative code paths that the test suite compares
// against the default ones (per-thread loads instead of bulk tensor copies,
// stream launches instead of graph replay) and host- or device-side failure
// hooks that need no GPU fault (an allocation that reports out-of-memory, a
// copy wait that is made to run out).  Their initial value comes from the
// environment, read once when the library is loaded; afterwards only
// disc_set_test_switches changes them.  Launch paths read one atomic word.

#include <atomic>
#include <cstdlib>

#include "internal.cuh"

namespace {

bool env_on(const char* name) {
  const char* v = std::getenv(name);
  return v != nullptr && v[0] != '\0' && v[0] != '0';
}

uint32_t env_switches() {
  uint32_t f = 0;
  if (env_on("DISC_NO_TMA")) f |= DISC_SW_NO_TMA;
  if (env_on("DISC_TEST_TMA_STALL")) f |= DISC_SW_TMA_STALL;
  if (env_on("DISC_NO_GRAPH")) f |= DISC_SW_NO_GRAPH;
  if (env_on("DISC_UNROLLED_GRAPH")) f |= DISC_SW_UNROLLED_GRAPH;
  if (env_on("DISC_WIDE_ANY")) f |= DISC_SW_WIDE_ANY;
  if (env_on("DISC_SEPARATE_WARP")) f |= DISC_SW_SEPARATE_WARP;
  if (env_on("DISC_FUSED_WARP")) f |= DISC_SW_FUSED_WARP;
  const char* fault = std::getenv("DISC_FAULT");
  if (fault != nullptr && fault[0] == 'a' && fault[1] == 'l' && fault[2] == 'l' && fault[3] == 'o' &&
      fault[4] == 'c' && fault[5] == '\0')
    f |= DISC_SW_FAULT_ALLOC;
  return f;
}

// initialised during the library's static initialisation (dlopen)
std::atomic<uint32_t> g_switches{env_switches()};

}  // namespace

namespace disc {

uint32_t test_switches() { return g_switches.load(std::memory_order_relaxed); }

}  // namespace disc

extern "C" disc_status disc_set_test_switches(uint32_t flags, uint32_t* previous) {
  if ((flags & ~(uint32_t)DISC_SW_ALL) != 0u) return DISC_ERR_ARG;
  const uint32_t old = g_switches.exchange(flags, std::memory_order_relaxed);
  if (previous) *previous = old;
  return DISC_OK;
}

// ---- bounds-checked build -----------------------------------------------------
#ifdef DISC_BOUNDS_CHECK
namespace disc {
__device__ unsigned long long g_bounds_violations = 0;
}
#endif

extern "C" disc_status disc_bounds_violations(void* stream, int64_t* count, int32_t* checked_build) {
  if (!count) return DISC_ERR_ARG;
  *count = 0;
#ifdef DISC_BOUNDS_CHECK
  if (checked_build) *checked_build = 1;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long* dev = nullptr;
  unsigned long long v = 0;
  cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&dev), disc::g_bounds_violations);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&v, dev, sizeof(v), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && v != 0) e = cudaMemsetAsync(dev, 0, sizeof(v), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return DISC_ERR_CUDA;
  }
  *count = (int64_t)v;
#else
  (void)stream;
  if (checked_build) *checked_build = 0;
#endif
  return DISC_OK;
}

