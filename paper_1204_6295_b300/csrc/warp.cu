// Trilinear warp of the moving image (Sec. 2.1, I_m(x + v(x)); Sec. 2.3
// kernel 5), sm_103a: m(x) = I_m(x + r(x)), sample position clamped to the
// volume.  One thread per voxel, x-contiguous, so that the field loads and the
// output store are coalesced and the eight taps of neighbouring threads share
// cache lines.

#include "internal.cuh"
#include "warp_dev.cuh"

namespace disc {

namespace {
constexpr int kWarpThreads = 128;

__global__ void __launch_bounds__(kWarpThreads) k_warp(const float* __restrict__ Im, const float* __restrict__ r,
                                                       float* __restrict__ m, int nx, int ny, int nz,
                                                       const int* stop) {
  if (stop != nullptr && *(volatile const int*)stop != 0) return;
  const int x = blockIdx.x * kWarpThreads + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  if (x >= nx) return;
  const size_t N = (size_t)nx * ny * nz;
  const size_t g = ((size_t)z * ny + y) * nx + x;
  m[g] = warp_at(Im, x, y, z, __ldg(r + g), __ldg(r + N + g), __ldg(r + 2 * N + g), nx, ny, nz);
}
}  // namespace

cudaError_t launch_warp(const float* Im, const float* r, float* m, int nx, int ny, int nz, const int* stop,
                        cudaStream_t s) {
  if (ny > 65535 || nz > 65535) return cudaErrorInvalidConfiguration;
  dim3 grid((nx + kWarpThreads - 1) / kWarpThreads, ny, nz);
  k_warp<<<grid, kWarpThreads, 0, s>>>(Im, r, m, nx, ny, nz, stop);
  return cudaGetLastError();
}

}  // namespace disc
