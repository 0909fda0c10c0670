// Gaussian regularisation of the displacement field (Algorithm A1 step 6;
// Sec. 2.3 kernel 2), sm_103a.
//
// r = G_sigma * u for each of the three field components, separable: taps
// w_i proportional to exp(-i^2 / 2 sigma^2), |i| <= R, and on each axis the
// weights are renormalised over the taps that fall inside the volume.
//
// A CTA owns a TX x TY column tile and marches over a chunk of z planes.  Each
// plane of u (3 components, tile plus R halo) is staged in shared memory,
// filtered along x and then y, and the xy-filtered plane is kept in a ring of
// 2R+1 planes from which the z filter emits the output plane R behind.

#include <cmath>

#include "internal.cuh"

namespace disc {

namespace {
constexpr int kGX = 32;
constexpr int kGY = 16;
constexpr size_t kMaxSmem = 226 * 1024;   // leaves room for the static tap buffer
constexpr int kMaxDevices = 64;
int g_smem_set[kMaxDevices] = {};

struct GaussLayout {
  int IX, IY, KZ;
  size_t o_in, o_xc, o_ring, total;
};

__host__ __device__ inline GaussLayout gauss_layout(int R) {
  GaussLayout L;
  L.IX = kGX + 2 * R;
  L.IY = kGY + 2 * R;
  L.KZ = 2 * R + 1;
  size_t o = 0;
  L.o_in = o;   o += 4 * 3 * (size_t)L.IX * L.IY;
  L.o_xc = o;   o += 4 * 3 * (size_t)kGX * L.IY;
  L.o_ring = o; o += 4 * 3 * (size_t)L.KZ * kGX * kGY;
  L.total = (o + 15) & ~(size_t)15;
  return L;
}

// Sum of the taps that land inside [0, n) for position c (the renormaliser).
__device__ __forceinline__ float tap_norm(const float* w, int R, int c, int n) {
  if (c - R >= 0 && c + R < n) return 1.0f;
  float s = 0.0f;
  for (int k = -R; k <= R; ++k)
    if (c + k >= 0 && c + k < n) s += w[k + R];
  return s;
}

__global__ void __launch_bounds__(kThreads) k_gauss(GaussArgs a) {
  if (a.stop != nullptr && *(volatile const int*)a.stop != 0) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const int R = a.R;
  const GaussLayout L = gauss_layout(R);
  float* in = reinterpret_cast<float*>(smem + L.o_in);
  float* xc = reinterpret_cast<float*>(smem + L.o_xc);
  float* ring = reinterpret_cast<float*>(smem + L.o_ring);
  __shared__ float w[2 * DISC_MAX_GAUSS_RADIUS + 1];
  const int tid = threadIdx.x;
  for (int k = tid; k < 2 * R + 1; k += kThreads) w[k] = a.w[k];

  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const size_t N = (size_t)nx * ny * nz;
  const int x0 = blockIdx.x * kGX, y0 = blockIdx.y * kGY;
  const int z0 = blockIdx.z * a.zlen;
  const int z1 = min(nz, z0 + a.zlen);
  const int IX = L.IX, IY = L.IY, KZ = L.KZ;
  const int INP = IX * IY, XCP = kGX * IY, OP = kGX * kGY;
  __syncthreads();

  const int zi0 = max(0, z0 - R);
  const int zi1 = z1 - 1 + R;
  for (int zi = zi0; zi <= zi1; ++zi) {
    if (zi < nz) {
      // stage the plane of u with its xy halo (zeros outside the volume)
      for (int e = tid; e < 3 * INP; e += kThreads) {
        const int c = e / INP, rem = e - c * INP;
        const int iy = rem / IX, ix = rem - iy * IX;
        const int gx = x0 - R + ix, gy = y0 - R + iy;
        float v = 0.0f;
        if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) v = __ldg(a.u + c * N + vix(gx, gy, zi, nx, ny));
        in[e] = v;
      }
      __syncthreads();
      // x filter
      for (int e = tid; e < 3 * XCP; e += kThreads) {
        const int c = e / XCP, rem = e - c * XCP;
        const int iy = rem / kGX, ox = rem - iy * kGX;
        const int gx = x0 + ox;
        if (gx >= nx) continue;
        const float* row = in + c * INP + iy * IX + ox;
        float acc = 0.0f;
        for (int k = 0; k <= 2 * R; ++k) acc = fmaf(w[k], row[k], acc);
        const float nrm = tap_norm(w, R, gx, nx);
        xc[e] = nrm == 1.0f ? acc : acc / nrm;
      }
      __syncthreads();
      // y filter into the z ring
      float* slot = ring + (zi % KZ) * 3 * OP;
      for (int e = tid; e < 3 * OP; e += kThreads) {
        const int c = e / OP, rem = e - c * OP;
        const int oy = rem / kGX, ox = rem - oy * kGX;
        const int gx = x0 + ox, gy = y0 + oy;
        if (gx >= nx || gy >= ny) continue;
        const float* col = xc + c * XCP + oy * kGX + ox;
        float acc = 0.0f;
        for (int k = 0; k <= 2 * R; ++k) acc = fmaf(w[k], col[k * kGX], acc);
        const float nrm = tap_norm(w, R, gy, ny);
        slot[e] = nrm == 1.0f ? acc : acc / nrm;
      }
      __syncthreads();
    }
    // z filter for the plane R behind
    const int zo = zi - R;
    if (zo >= z0 && zo < z1) {
      const float nrm = tap_norm(w, R, zo, nz);
      const int klo = max(-R, -zo), khi = min(R, nz - 1 - zo);
      for (int e = tid; e < 3 * OP; e += kThreads) {
        const int c = e / OP, rem = e - c * OP;
        const int oy = rem / kGX, ox = rem - oy * kGX;
        const int gx = x0 + ox, gy = y0 + oy;
        if (gx >= nx || gy >= ny) continue;
        float acc = 0.0f;
        for (int k = klo; k <= khi; ++k) acc = fmaf(w[k + R], ring[((zo + k) % KZ) * 3 * OP + e], acc);
        a.r[c * N + vix(gx, gy, zo, nx, ny)] = nrm == 1.0f ? acc : acc / nrm;
      }
    }
  }
}
}  // namespace

int gauss_radius(float sigma, int radius) {
  if (radius > 0) return radius;
  return (int)std::ceil(3.0 * (double)sigma);
}

void gauss_taps(float sigma, int R, float* w) {
  double t[2 * DISC_MAX_GAUSS_RADIUS + 1];
  double s = 0.0;
  for (int k = -R; k <= R; ++k) {
    t[k + R] = std::exp(-(double)k * k / (2.0 * (double)sigma * sigma));
    s += t[k + R];
  }
  for (int k = 0; k <= 2 * R; ++k) w[k] = (float)(t[k] / s);
}

GaussPlan gauss_plan(int nx, int ny, int nz, int R, int num_sms) {
  GaussPlan p;
  const GaussLayout L = gauss_layout(R);
  p.smem = L.total;
  if (p.smem > kMaxSmem) {
    p.grid = dim3(0, 0, 0);
    p.zlen = 0;
    return p;
  }
  const int gx = (nx + kGX - 1) / kGX, gy = (ny + kGY - 1) / kGY;
  int per_sm = (int)(kMaxSmem / (p.smem + 1024));
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 8) per_sm = 8;
  const long long target = 2LL * num_sms * per_sm;
  long long chunks = (target + (long long)gx * gy - 1) / ((long long)gx * gy);
  if (chunks < 1) chunks = 1;
  long long max_chunks = (nz + 3) / 4;
  if (max_chunks < 1) max_chunks = 1;
  if (chunks > max_chunks) chunks = max_chunks;
  p.zlen = (int)((nz + chunks - 1) / chunks);
  p.grid = dim3(gx, gy, (nz + p.zlen - 1) / p.zlen);
  return p;
}

cudaError_t gauss_launch(const GaussArgs& a, const GaussPlan& p, cudaStream_t s) {
  if (p.grid.x == 0) return cudaErrorInvalidConfiguration;
  GaussArgs b = a;
  b.zlen = p.zlen;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  if ((int)p.smem > g_smem_set[dev]) {
    e = cudaFuncSetAttribute(k_gauss, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
    if (e != cudaSuccess) return e;
    g_smem_set[dev] = (int)kMaxSmem;
  }
  k_gauss<<<p.grid, kThreads, p.smem, s>>>(b);
  return cudaGetLastError();
}

}  // namespace disc
