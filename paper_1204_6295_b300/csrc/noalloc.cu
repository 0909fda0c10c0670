// disc_k_pass_a_static: the iteration front of disc_k_pass_a without any
// device allocation.
//
// disc_k_pass_a takes its per-CTA norm partials (and, when the caller passes no
// m buffer, the warped image) from the stream-ordered allocator.  Some callers
// cannot let a library allocate device memory at all: applications that own
// every byte of device memory through their own pool or run under a fixed
// memory budget, and hosts that forbid plug-in libraries from calling
// cudaMalloc or the stream-ordered allocator.  This entry point keeps its only
// scratch, the per-CTA partial sums, in a file-scope __device__ array of fixed
// size, and requires the caller to pass the warped-image buffer as an output.
//
// The array lives in every device that loads this library, for the life of the
// process.  Host code cannot pass the array's name to a kernel (on the host it
// names a host-side stand-in, not device memory), so the first call on each
// device looks its device address up with cudaGetSymbolAddress while that
// device is current, and caches it for the life of the process.  That first
// call should therefore come before any stream capture.  The cache is never
// invalidated: after cudaDeviceReset the device's module (and the array) is
// loaded anew, possibly elsewhere, so a process that resets a device must not
// call this entry point on it again.  Every call shares the one array: two calls whose
// work overlaps on the GPU race on it.  Each launch overwrites every partial it
// later reads, so nothing needs clearing between calls.

#include <mutex>

#include "internal.cuh"

using namespace disc;

namespace {

// Largest launch grid (CTAs) this entry point accepts: one float2 of partials
// per CTA, 64 KiB in total.
constexpr int kStaticPartials = 8192;
static __device__ __align__(256) float g_pass_a_partials[2 * kStaticPartials];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float* g_addr[kMaxDevices] = {};

// Device address of g_pass_a_partials on the current device (looked up once per device).
cudaError_t partials_address(float** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_addr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_pass_a_partials);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<float*>(p);
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" disc_status disc_k_pass_a_static(const float* Im, const float* zs, const float* r, float* u,
                                            float* m_out, float* d_out, double* norms_out, int32_t nx,
                                            int32_t ny, int32_t nz, const int32_t patch[3], float qscale,
                                            float var_floor, int32_t force_mode, void* stream) {
  if (!Im || !zs || !r || !u || !m_out || !patch || !(qscale > 0.0f) || !(var_floor >= 0.0f))
    return DISC_ERR_ARG;
  if (u == r) return DISC_ERR_ARG;
  if (force_mode != DISC_FORCE_THIRION && force_mode != DISC_FORCE_DOUBLE) return DISC_ERR_ARG;
  int h[3];
  for (int a = 0; a < 3; ++a) {
    if (patch[a] < 1 || patch[a] > 2 * DISC_MAX_HALF_PATCH + 1 || patch[a] % 2 == 0) return DISC_ERR_ARG;
    h[a] = (patch[a] - 1) / 2;
  }
  if (nx < 1 || ny < 1 || nz < 1 || ny > 65535 || nz > 65535) return DISC_ERR_SHAPE;
  int dev = 0, sms = kNumSMs;
  if (cudaGetDevice(&dev) != cudaSuccess) return DISC_ERR_CUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const BoxPlan p = box_plan(kModeIterate, nx, ny, nz, h[0], h[1], h[2], sms);
  if (p.grid.x == 0) return DISC_ERR_SHAPE;
  const long long nparts = (long long)p.grid.x * p.grid.y * p.grid.z;
  if (nparts > kStaticPartials) return DISC_ERR_SHAPE;   // beyond the fixed scratch
  float* parts = nullptr;
  if (partials_address(&parts) != cudaSuccess) {
    cudaGetLastError();
    return DISC_ERR_CUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = launch_warp(Im, r, m_out, nx, ny, nz, nullptr, s);
  BoxArgs a{};
  a.src = m_out;
  a.zs = zs;
  a.r = r;
  a.out = u;
  a.f_tap = d_out;
  a.partials = parts;
  a.nx = nx;
  a.ny = ny;
  a.nz = nz;
  a.hx = h[0];
  a.hy = h[1];
  a.hz = h[2];
  a.qscale = qscale;
  a.inv_qscale = 1.0f / qscale;
  a.var_floor = var_floor;
  a.force_mode = force_mode;
  if (e == cudaSuccess) e = box_launch(kModeIterate, a, p, s);
  if (e == cudaSuccess && norms_out) {
    e = launch_partials_sum(parts, (int)nparts, 0, norms_out, s);
    if (e == cudaSuccess) e = launch_partials_sum(parts, (int)nparts, 1, norms_out + 1, s);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return DISC_ERR_CUDA;
  }
  return DISC_OK;
}
