// Trilinear sampling of the moving image, shared by the warp kernel and the
// fused Gaussian z pass: m(x) = I_m(x + r(x)) with the sample position clamped
// to the volume (Sec. 2.1; Sec. 2.3 kernel 5).
#pragma once

#include <cuda_runtime.h>

namespace disc {

// Sample position along one axis: voxel c displaced by rv, clamped to
// [0, n-1].  The integer part is formed as c + floor(rv) so that the fraction
// rv - floor(rv) does not depend on the voxel's position.
static __device__ __forceinline__ void axis_setup(int c, float rv, int n, int& i0, int& i1, float& t) {
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

static __device__ __forceinline__ float lerpf(float a, float b, float t) { return fmaf(t, b - a, a); }

static __device__ __forceinline__ float warp_at(const float* __restrict__ Im, int x, int y, int z, float rx,
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

}  // namespace disc
