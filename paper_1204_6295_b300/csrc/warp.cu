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
// z-marching form: a thread owns one (x, y) column of a chunk of planes and
// loads the field of plane z + kWarpAhead while it gathers I_m for plane z, so
// that the field's trip to memory overlaps the gathers instead of preceding
// them (the two are otherwise dependent round trips per voxel).  CTAs of 32 x 4
// columns: a warp's field loads and m stores are coalesced rows, and its rows'
// gathers share cache lines.
constexpr int kWarpZX = 32, kWarpZY = 4, kWarpAhead = 2, kWarpZChunk = 16;
// Column (x, y) of CTA (bx, by), planes [bz kWarpZChunk, (bz + 1) kWarpZChunk).
// The field and image indices fit 32 bits (3 N < 2^31, checked by the launch).
__device__ __forceinline__ void warp_z_body(const float* __restrict__ Im, const float* __restrict__ r,
                                            float* __restrict__ m, int nx, int ny, int nz, int bx, int by,
                                            int bz) {
  const int x = bx * kWarpZX + threadIdx.x % kWarpZX;
  const int y = by * kWarpZY + threadIdx.x / kWarpZX;
  if (x >= nx || y >= ny) return;
  const int z0 = bz * kWarpZChunk, z1 = min(nz, z0 + kWarpZChunk);
  const int plane = nx * ny, N = plane * nz;
  const int col = y * nx + x;
  float rq[kWarpAhead + 1][3];
#pragma unroll
  for (int k = 0; k < kWarpAhead; ++k) {
    const int z = z0 + k;
    if (z < z1) {
      const int g = z * plane + col;
      rq[k][0] = ldcs_in(r, g, 3LL * N);
      rq[k][1] = ldcs_in(r, N + g, 3LL * N);
      rq[k][2] = ldcs_in(r, 2 * N + g, 3LL * N);
    }
  }
  for (int zb = z0; zb < z1; zb += kWarpAhead + 1) {
#pragma unroll
    for (int j = 0; j <= kWarpAhead; ++j) {   // slots rotate with z: the unrolled loop keeps them static
      const int z = zb + j;
      if (z >= z1) break;
      const int zn = z + kWarpAhead;          // the plane whose field is loaded now
      const int sn = (j + kWarpAhead) % (kWarpAhead + 1);
      if (zn < z1) {
        const int g = zn * plane + col;
        rq[sn][0] = ldcs_in(r, g, 3LL * N);
        rq[sn][1] = ldcs_in(r, N + g, 3LL * N);
        rq[sn][2] = ldcs_in(r, 2 * N + g, 3LL * N);
      }
      st_in(m, z * plane + col, (long long)N, warp_at32(Im, x, y, z, rq[j][0], rq[j][1], rq[j][2], nx, ny, nz));
    }
  }
}

__global__ void __launch_bounds__(kWarpZX * kWarpZY) k_warp_z(const float* __restrict__ Im, const float* __restrict__ r,
                                                               float* __restrict__ m, int nx, int ny, int nz,
                                                               const int* stop) {
  pdl_wait();
  pdl_release();
  if (stop != nullptr && *(volatile const int*)stop != 0) return;
  warp_z_body(Im, r, m, nx, ny, nz, blockIdx.x, blockIdx.y, blockIdx.z);
}

// Batched z-marching warp: CTA i runs block i - offset[p] of pair p's grid
// (warp_z_blocks of its volume, x fastest).
__global__ void __launch_bounds__(kWarpZX * kWarpZY) k_warp_z_batch(const __grid_constant__ WarpBatch wb) {
  pdl_wait();
  pdl_release();
  const int i = blockIdx.x;
  int p = 0;
  while (p + 1 < wb.count && wb.offset[p + 1] <= i) ++p;
  if (wb.stop[p] != nullptr && *(volatile const int*)wb.stop[p] != 0) return;
  const int nx = wb.nx[p], ny = wb.ny[p];
  const int gx = (nx + kWarpZX - 1) / kWarpZX, gy = (ny + kWarpZY - 1) / kWarpZY;
  const int j = i - wb.offset[p];
  warp_z_body(wb.Im[p], wb.r[p], wb.m[p], nx, ny, wb.nz[p], j % gx, (j / gx) % gy, j / (gx * gy));
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

int warp_z_blocks(int nx, int ny, int nz) {
  return ((nx + kWarpZX - 1) / kWarpZX) * ((ny + kWarpZY - 1) / kWarpZY) * ((nz + kWarpZChunk - 1) / kWarpZChunk);
}

cudaError_t launch_warp_z_batch(const WarpBatch& wb, int total_blocks, cudaStream_t s) {
  if (total_blocks < 1) return cudaSuccess;
  return launch_pdl(k_warp_z_batch, dim3(total_blocks), dim3(kWarpZX * kWarpZY), 0, s, wb);
}

cudaError_t launch_warp(const float* Im, const float* r, float* m, int nx, int ny, int nz, const int* stop,
                        cudaStream_t s) {
  if (ny > 65535 || nz > 65535) return cudaErrorInvalidConfiguration;
  if (nx >= kWarpZX && nz >= kWarpZChunk && 3.0 * nx * ny * nz < 2147483647.0) {
    dim3 grid((nx + kWarpZX - 1) / kWarpZX, (ny + kWarpZY - 1) / kWarpZY, (nz + kWarpZChunk - 1) / kWarpZChunk);
    return launch_pdl(k_warp_z, grid, dim3(kWarpZX * kWarpZY), 0, s, Im, r, m, nx, ny, nz, stop);
  }
  dim3 grid((nx + kWarpThreads - 1) / kWarpThreads, ny, nz);
  k_warp<<<grid, kWarpThreads, 0, s>>>(Im, r, m, nx, ny, nz, stop);
  return cudaGetLastError();
}

}  // namespace disc
