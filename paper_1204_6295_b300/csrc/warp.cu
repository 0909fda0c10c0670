// Trilinear warp of the moving image (Sec. 2.1, I_m(x + v(x)); Sec. 2.3
// kernel 5), sm_103a: m(x) = I_m(x + r(x)), sample position clamped to the
// volume.  One thread per voxel, x-contiguous, so that the field loads and the
// output store are coalesced and the eight taps of neighbouring threads share
// cache lines.

#include "internal.cuh"

namespace disc {

// Sample position along one axis: voxel c displaced by rv, clamped to
// [0, n-1].  The integer part is formed as c + floor(rv) so that the fraction
// rv - floor(rv) does not depend on the voxel's position.
__device__ __forceinline__ void axis_setup(int c, float rv, int n, int& i0, int& i1, float& t) {
  float fl = floorf(rv);
  fl = fminf(fmaxf(fl, -1073741824.0f), 1073741824.0f);   // also maps NaN to a clamp
  int i = c + (int)fl;
  t = rv - fl;
  if (i < 0) {
    i = 0;
    t = 0.0f;
  } else if (i >= n - 1) {
    i = n - 1;
    t = 0.0f;
  }
  i0 = i;
  i1 = min(i + 1, n - 1);
}

__device__ __forceinline__ float lerpf(float a, float b, float t) { return fmaf(t, b - a, a); }

__device__ __forceinline__ float warp_at(const float* __restrict__ Im, int x, int y, int z, float rx,
                                         float ry, float rz, int nx, int ny, int nz) {
  int x0, x1, y0, y1, z0, z1;
  float tx, ty, tz;
  axis_setup(x, rx, nx, x0, x1, tx);
  axis_setup(y, ry, ny, y0, y1, ty);
  axis_setup(z, rz, nz, z0, z1, tz);
  const size_t sy0 = (size_t)y0 * nx, sy1 = (size_t)y1 * nx;
  const size_t sz0 = (size_t)z0 * ny * nx, sz1 = (size_t)z1 * ny * nx;
  const float c000 = __ldg(Im + sz0 + sy0 + x0), c001 = __ldg(Im + sz0 + sy0 + x1);
  const float c010 = __ldg(Im + sz0 + sy1 + x0), c011 = __ldg(Im + sz0 + sy1 + x1);
  const float c100 = __ldg(Im + sz1 + sy0 + x0), c101 = __ldg(Im + sz1 + sy0 + x1);
  const float c110 = __ldg(Im + sz1 + sy1 + x0), c111 = __ldg(Im + sz1 + sy1 + x1);
  const float c00 = lerpf(c000, c001, tx), c01 = lerpf(c010, c011, tx);
  const float c10 = lerpf(c100, c101, tx), c11 = lerpf(c110, c111, tx);
  return lerpf(lerpf(c00, c01, ty), lerpf(c10, c11, ty), tz);
}

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
