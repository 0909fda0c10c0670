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
  st_in(m, g, N,
        warp_at(Im, x, y, z, ldg_in(r, g, 3 * N), ldg_in(r, N + g, 3 * N), ldg_in(r, 2 * N + g, 3 * N), nx, ny,
                nz));
}
}  // namespace

__global__ void __launch_bounds__(kWarpBatchThreads) k_warp_batch(const __grid_constant__ WarpBatch wb) {
  const int i = blockIdx.x;
  int p = 0;
  while (p + 1 < wb.count && wb.offset[p + 1] <= i) ++p;
  if (wb.stop[p] != nullptr && *(volatile const int*)wb.stop[p] != 0) return;
  const int nx = wb.nx[p], ny = wb.ny[p], nz = wb.nz[p];
  const int j = i - wb.offset[p];
  const int gxb = (nx + kWarpBatchThreads - 1) / kWarpBatchThreads;
  const int x = (j % gxb) * kWarpBatchThreads + threadIdx.x;
  const int y = (j / gxb) % ny, z = j / (gxb * ny);
  if (x >= nx) return;
  const size_t N = (size_t)nx * ny * nz;
  const size_t g = ((size_t)z * ny + y) * nx + x;
  const float* r = wb.r[p];
  st_in(wb.m[p], g, N,
        warp_at(wb.Im[p], x, y, z, ldg_in(r, g, 3 * N), ldg_in(r, N + g, 3 * N), ldg_in(r, 2 * N + g, 3 * N), nx,
                ny, nz));
}

cudaError_t launch_warp_batch(const WarpBatch& wb, int total_blocks, cudaStream_t s) {
  if (total_blocks < 1) return cudaSuccess;
  k_warp_batch<<<total_blocks, kWarpBatchThreads, 0, s>>>(wb);
  return cudaGetLastError();
}

cudaError_t launch_warp(const float* Im, const float* r, float* m, int nx, int ny, int nz, const int* stop,
                        cudaStream_t s) {
  if (ny > 65535 || nz > 65535) return cudaErrorInvalidConfiguration;
  dim3 grid((nx + kWarpThreads - 1) / kWarpThreads, ny, nz);
  k_warp<<<grid, kWarpThreads, 0, s>>>(Im, r, m, nx, ny, nz, stop);
  return cudaGetLastError();
}

}  // namespace disc
