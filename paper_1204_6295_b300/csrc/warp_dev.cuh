// Trilinear sampling of the moving image, shared by the warp kernel and the
// fused Gaussian xy pass: m(x) = I_m(x + r(x)) with the sample position clamped
// to the volume (Sec. 2.1; Sec. 2.3 kernel 5).
#pragma once

#include <cuda_runtime.h>

#include "internal.cuh"

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

// warp_at for volumes of fewer than 2^31 voxels: the eight sample indices in
// 32-bit arithmetic (one wide address computation per gather).  Same samples,
// same interpolation, same bits.
static __device__ __forceinline__ float warp_at32(const float* __restrict__ Im, int x, int y, int z, float rx,
                                                  float ry, float rz, int nx, int ny, int nz) {
  int x0, x1, y0, y1, z0, z1;
  float tx, ty, tz;
  axis_setup(x, rx, nx, x0, x1, tx);
  axis_setup(y, ry, ny, y0, y1, ty);
  axis_setup(z, rz, nz, z0, z1, tz);
  const int plane = nx * ny;
  const int b00 = z0 * plane + y0 * nx, b01 = z0 * plane + y1 * nx;
  const int b10 = z1 * plane + y0 * nx, b11 = z1 * plane + y1 * nx;
#ifdef DISC_BOUNDS_CHECK
  const long long n = (long long)plane * nz;
  auto ld = [&](int i) { return DISC_IN(i, n) ? __ldg(Im + i) : 0.0f; };
#else
  auto ld = [&](int i) { return __ldg(Im + i); };
#endif
  const float c000 = ld(b00 + x0), c001 = ld(b00 + x1);
  const float c010 = ld(b01 + x0), c011 = ld(b01 + x1);
  const float c100 = ld(b10 + x0), c101 = ld(b10 + x1);
  const float c110 = ld(b11 + x0), c111 = ld(b11 + x1);
  const float c00 = lerpf(c000, c001, tx), c01 = lerpf(c010, c011, tx);
  const float c10 = lerpf(c100, c101, tx), c11 = lerpf(c110, c111, tx);
  return lerpf(lerpf(c00, c01, ty), lerpf(c10, c11, ty), tz);
}

static __device__ __forceinline__ float warp_at(const float* __restrict__ Im, int x, int y, int z, float rx,
                                         float ry, float rz, int nx, int ny, int nz) {
  int x0, x1, y0, y1, z0, z1;
  float tx, ty, tz;
  axis_setup(x, rx, nx, x0, x1, tx);
  axis_setup(y, ry, ny, y0, y1, ty);
  axis_setup(z, rz, nz, z0, z1, tz);
  const size_t sy0 = (size_t)y0 * nx, sy1 = (size_t)y1 * nx;
  const size_t sz0 = (size_t)z0 * ny * nx, sz1 = (size_t)z1 * ny * nx;
#ifdef DISC_BOUNDS_CHECK
  const long long n = (long long)nx * ny * nz;
  auto ld = [&](size_t i) { return DISC_IN(i, n) ? __ldg(Im + i) : 0.0f; };
#else
  auto ld = [&](size_t i) { return __ldg(Im + i); };
#endif
  const float c000 = ld(sz0 + sy0 + x0), c001 = ld(sz0 + sy0 + x1);
  const float c010 = ld(sz0 + sy1 + x0), c011 = ld(sz0 + sy1 + x1);
  const float c100 = ld(sz1 + sy0 + x0), c101 = ld(sz1 + sy0 + x1);
  const float c110 = ld(sz1 + sy1 + x0), c111 = ld(sz1 + sy1 + x1);
  const float c00 = lerpf(c000, c001, tx), c01 = lerpf(c010, c011, tx);
  const float c10 = lerpf(c100, c101, tx), c11 = lerpf(c110, c111, tx);
  return lerpf(lerpf(c00, c01, ty), lerpf(c10, c11, ty), tz);
}


// d I_m(p) / d p at p = (x, y, z) + r for the trilinear interpolant, with the
// cell chosen as in warp_at ([floor(p), floor(p) + 1]); zero along an axis whose
// sample position is clamped (p <= 0 or p >= n - 1 before clamping).
static __device__ __forceinline__ void warp_grad_at(const float* __restrict__ Im, int x, int y, int z,
                                                    float rx, float ry, float rz, int nx, int ny, int nz,
                                                    float& gx, float& gy, float& gz) {
  int i0[3], i1[3];
  float t[3];
  bool inside[3];
  const int c[3] = {x, y, z};
  const float rv[3] = {rx, ry, rz};
  const int n[3] = {nx, ny, nz};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float fl = floorf(rv[a]);
    fl = fminf(fmaxf(fl, -1073741824.0f), 1073741824.0f);
    const int i = c[a] + (int)fl;
    const float tt = rv[a] - fl;
    inside[a] = (i > 0 || (i == 0 && tt > 0.0f)) && i <= n[a] - 2;
    axis_setup(c[a], rv[a], n[a], i0[a], i1[a], t[a]);
  }
  const size_t sx = 1, sy = (size_t)nx, sz = (size_t)nx * ny;
  auto at = [&](int a, int b, int cc) {
    const size_t i = (size_t)cc * sz + (size_t)b * sy + (size_t)a * sx;
    return DISC_IN(i, (long long)nx * ny * nz) ? __ldg(Im + i) : 0.0f;
  };
  const float c000 = at(i0[0], i0[1], i0[2]), c100 = at(i1[0], i0[1], i0[2]);
  const float c010 = at(i0[0], i1[1], i0[2]), c110 = at(i1[0], i1[1], i0[2]);
  const float c001 = at(i0[0], i0[1], i1[2]), c101 = at(i1[0], i0[1], i1[2]);
  const float c011 = at(i0[0], i1[1], i1[2]), c111 = at(i1[0], i1[1], i1[2]);
  const float tx = t[0], ty = t[1], tz = t[2];
  // d/dx: differences along x, interpolated in y and z
  const float dx00 = c100 - c000, dx10 = c110 - c010, dx01 = c101 - c001, dx11 = c111 - c011;
  const float dy00 = c010 - c000, dy10 = c110 - c100, dy01 = c011 - c001, dy11 = c111 - c101;
  const float dz00 = c001 - c000, dz10 = c101 - c100, dz01 = c011 - c010, dz11 = c111 - c110;
  gx = inside[0] ? lerpf(lerpf(dx00, dx10, ty), lerpf(dx01, dx11, ty), tz) : 0.0f;
  gy = inside[1] ? lerpf(lerpf(dy00, dy10, tx), lerpf(dy01, dy11, tx), tz) : 0.0f;
  gz = inside[2] ? lerpf(lerpf(dz00, dz10, tx), lerpf(dz01, dz11, tx), ty) : 0.0f;
}

}  // namespace disc
