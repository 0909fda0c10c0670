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
// Four x-consecutive voxels per thread (nx a multiple of 4, 16-byte aligned
// buffers): the field is read and m written as 16-byte vectors, and the 32
// gathers of a thread are independent, so more of them are in flight.
constexpr int kWarp4Threads = 128;
__global__ void __launch_bounds__(kWarp4Threads) k_warp4(const float* __restrict__ Im, const float* __restrict__ r,
                                                         float* __restrict__ m, int nx, int ny, int nz,
                                                         const int* stop) {
  pdl_wait();
  pdl_release();
  if (stop != nullptr && *(volatile const int*)stop != 0) return;
  const int x = 4 * (blockIdx.x * kWarp4Threads + threadIdx.x);
  const int y = blockIdx.y, z = blockIdx.z;
  if (x >= nx) return;
  const long long N = (long long)nx * ny * nz;
  const long long q = (((long long)z * ny + y) * nx + x) / 4;   // float4 index
  const float4* r4 = reinterpret_cast<const float4*>(r);
  const float4 rx = ldg_in(r4, q, 3 * (N / 4)), ry = ldg_in(r4, q + N / 4, 3 * (N / 4));
  const float4 rz = ldg_in(r4, q + 2 * (N / 4), 3 * (N / 4));
  float4 o;
  o.x = warp_at(Im, x, y, z, rx.x, ry.x, rz.x, nx, ny, nz);
  o.y = warp_at(Im, x + 1, y, z, rx.y, ry.y, rz.y, nx, ny, nz);
  o.z = warp_at(Im, x + 2, y, z, rx.z, ry.z, rz.z, nx, ny, nz);
  o.w = warp_at(Im, x + 3, y, z, rx.w, ry.w, rz.w, nx, ny, nz);
  st_in(reinterpret_cast<float4*>(m), q, N / 4, o);
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
  if (nx % 4 == 0 && (((uintptr_t)r | (uintptr_t)m) & 15u) == 0u) {
    dim3 grid((nx / 4 + kWarp4Threads - 1) / kWarp4Threads, ny, nz);
    return launch_pdl(k_warp4, grid, dim3(kWarp4Threads), 0, s, Im, r, m, nx, ny, nz, stop);
  }
  dim3 grid((nx + kWarpThreads - 1) / kWarpThreads, ny, nz);
  k_warp<<<grid, kWarpThreads, 0, s>>>(Im, r, m, nx, ny, nz, stop);
  return cudaGetLastError();
}

}  // namespace disc
