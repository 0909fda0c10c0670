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

// ---------------------------------------------------------------------------
// Register-queue form for radius R (compile time).  A CTA owns a 32 x 16
// tile; each thread owns two x-adjacent voxels of one row and all three field
// components.  Per plane: stage the plane (tile + R halo) in shared memory,
// filter along x into shared memory, then each thread filters its own column
// along y and adds the result, times each z tap, into a queue of 2R+1 pending
// output planes held in registers (float2, packed FFMA2).  The queue slot of
// output plane z is z mod (2R+1), made static by unrolling the plane loop by
// 2R+1.  The next plane's loads are issued before the y/z work of the
// current one, so their latency overlaps the arithmetic.
// ---------------------------------------------------------------------------
constexpr int kQX = 32;
constexpr int kQY = 16;

template <int R>
struct QLayout {
  static constexpr int IX = kQX + 2 * R;
  static constexpr int IY = kQY + 2 * R;
  static constexpr int KZ = 2 * R + 1;
  static constexpr int INP = IX * IY;          // floats per component plane
  static constexpr int XCP = (kQX / 2) * IY;   // float2 per component plane
  static constexpr int NLOAD = (3 * INP + kThreads - 1) / kThreads;
  static constexpr size_t o_ring = 0;
  static constexpr size_t o_xc = o_ring + 8 * (size_t)KZ * 3 * kThreads;
  static constexpr size_t o_in = o_xc + 8 * 3 * (size_t)XCP;
  static constexpr size_t bytes = o_in + 4 * 3 * (size_t)INP;
};

template <int R>
__global__ void __launch_bounds__(kThreads) k_gauss_q(GaussArgs a) {
  using Q = QLayout<R>;
  if (a.stop != nullptr && *(volatile const int*)a.stop != 0) return;
  extern __shared__ __align__(16) unsigned char smem[];
  float* in = reinterpret_cast<float*>(smem + Q::o_in);
  float2* xc = reinterpret_cast<float2*>(smem + Q::o_xc);
  float2* ring = reinterpret_cast<float2*>(smem + Q::o_ring);   // [KZ][3][threads], thread-private
  __shared__ float w[2 * R + 1];
  __shared__ float nrm_x[kQX], nrm_y[kQY];
  const int tid = threadIdx.x;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const size_t plane = (size_t)nx * ny;
  const size_t N = plane * nz;
  const int x0 = blockIdx.x * kQX, y0 = blockIdx.y * kQY;
  const int z0 = blockIdx.z * a.zlen;
  const int z1 = min(nz, z0 + a.zlen);
  if (tid < 2 * R + 1) w[tid] = a.w[tid];
#pragma unroll
  for (int j = 0; j < Q::KZ * 3; ++j) ring[j * kThreads + tid] = make_float2(0.0f, 0.0f);
  __syncthreads();
  if (tid < kQX) nrm_x[tid] = tap_norm(w, R, x0 + tid, nx);
  if (tid >= 64 && tid < 64 + kQY) nrm_y[tid - 64] = tap_norm(w, R, y0 + tid - 64, ny);

  // this thread's output pair
  const int px = tid & 15, oy = tid >> 4;
  const int gx = x0 + 2 * px, gy = y0 + oy;
  const bool own0 = gx < nx && gy < ny, own1 = gx + 1 < nx && gy < ny;

  // staged-plane element e -> global offset c N + Y nx + X (or -1 outside)
  int goff[Q::NLOAD];
#pragma unroll
  for (int k = 0; k < Q::NLOAD; ++k) {
    const int e = tid + k * kThreads;
    goff[k] = -1;
    if (e < 3 * Q::INP) {
      const int c = e / Q::INP, rem = e - c * Q::INP;
      const int iy = rem / Q::IX, ix = rem - iy * Q::IX;
      const int X = x0 - R + ix, Y = y0 - R + iy;
      if (X >= 0 && X < nx && Y >= 0 && Y < ny) goff[k] = (int)((size_t)c * N + (size_t)Y * nx + X);
    }
  }
  float pre[Q::NLOAD];
  const int zs = max(0, z0 - R);
  const int ze = z1 - 1 + R;                 // last plane that still feeds an output
  auto prefetch = [&](int z) {
#pragma unroll
    for (int k = 0; k < Q::NLOAD; ++k)
      pre[k] = (z < nz && goff[k] >= 0) ? __ldg(a.u + (size_t)goff[k] + (size_t)z * plane) : 0.0f;
  };

  prefetch(zs);
  __syncthreads();
  const float nyv = nrm_y[oy];
  for (int zi = zs; zi <= ze; ++zi) {
    const bool live = zi < nz;               // uniform
    float2* slot = ring + (zi % Q::KZ) * 3 * kThreads + tid;
    if (live) {
      __syncthreads();                       // the previous plane's y filter is done with xc
#pragma unroll
      for (int k = 0; k < Q::NLOAD; ++k) {
        const int e = tid + k * kThreads;
        if (e < 3 * Q::INP) in[e] = pre[k];
      }
      __syncthreads();
      // x filter: (component, row, pair) tasks
      for (int t = tid; t < 3 * Q::XCP; t += kThreads) {
        const int c = t / Q::XCP, rem = t - c * Q::XCP;
        const int iy = rem / (kQX / 2), jx = rem - iy * (kQX / 2);
        const float* row = in + c * Q::INP + iy * Q::IX + 2 * jx;
        float2 sacc = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int k = 0; k <= 2 * R; ++k)
          sacc = __ffma2_rn(make_float2(w[k], w[k]), make_float2(row[k], row[k + 1]), sacc);
        const float n0 = nrm_x[2 * jx], n1 = nrm_x[2 * jx + 1];
        if (n0 != 1.0f) sacc.x = sacc.x / n0;
        if (n1 != 1.0f) sacc.y = sacc.y / n1;
        xc[t] = sacc;
      }
      __syncthreads();
      if (zi + 1 <= ze) prefetch(zi + 1);    // overlaps the y/z work below
      // y filter of this thread's pair into its private ring slot
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float2* col = xc + c * Q::XCP + oy * (kQX / 2) + px;
        float2 t2 = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int k = 0; k <= 2 * R; ++k) t2 = __ffma2_rn(make_float2(w[k], w[k]), col[k * (kQX / 2)], t2);
        if (nyv != 1.0f) {
          t2.x = t2.x / nyv;
          t2.y = t2.y / nyv;
        }
        slot[c * kThreads] = t2;
      }
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c) slot[c * kThreads] = make_float2(0.0f, 0.0f);
      if (zi + 1 <= ze) prefetch(zi + 1);
    }
    // z filter for output plane zo = zi - R (planes outside the volume hold 0)
    const int zo = zi - R;
    if (zo >= z0 && zo < z1) {
      float2 o[3] = {make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)};
#pragma unroll
      for (int k = -R; k <= R; ++k) {
        const float2* sk = ring + ((zo + k + Q::KZ) % Q::KZ) * 3 * kThreads + tid;
        const float2 wk = make_float2(w[k + R], w[k + R]);
#pragma unroll
        for (int c = 0; c < 3; ++c) o[c] = __ffma2_rn(wk, sk[c * kThreads], o[c]);
      }
      const float nz_ = tap_norm(w, R, zo, nz);
      const size_t g = (size_t)zo * plane + (size_t)gy * nx + gx;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float2 oc = o[c];
        if (nz_ != 1.0f) {
          oc.x = oc.x / nz_;
          oc.y = oc.y / nz_;
        }
        if (own0) a.r[c * N + g] = oc.x;
        if (own1) a.r[c * N + g + 1] = oc.y;
      }
    }
  }
}

template <int R>
cudaError_t launch_q(const GaussArgs& a, const GaussPlan& p, cudaStream_t s) {
  static int set[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!set[dev]) {
    e = cudaFuncSetAttribute(k_gauss_q<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
    if (e != cudaSuccess) return e;
    set[dev] = 1;
  }
  k_gauss_q<R><<<p.grid, kThreads, p.smem, s>>>(a);
  return cudaGetLastError();
}

size_t q_smem(int R) {
  switch (R) {
#define QCASE(RR) case RR: return QLayout<RR>::bytes;
    QCASE(1) QCASE(2) QCASE(3) QCASE(4) QCASE(5) QCASE(6) QCASE(7) QCASE(8)
#undef QCASE
    default: return 0;
  }
}

cudaError_t launch_q_any(const GaussArgs& a, const GaussPlan& p, cudaStream_t s) {
  switch (a.R) {
#define QCASE(RR) case RR: return launch_q<RR>(a, p, s);
    QCASE(1) QCASE(2) QCASE(3) QCASE(4) QCASE(5) QCASE(6) QCASE(7) QCASE(8)
#undef QCASE
    default: return cudaErrorInvalidValue;
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
  p.queue = R >= 1 && R <= 8 && 3.0 * nx * ny * nz < 2147483647.0;
  if (p.queue) {
    p.smem = q_smem(R);
    const int gx = (nx + kQX - 1) / kQX, gy = (ny + kQY - 1) / kQY;
    int per_sm = (int)((228 * 1024) / (p.smem + 1024));
    if (per_sm < 1) per_sm = 1;
    if (per_sm > 3) per_sm = 3;
    const long long slots = (long long)num_sms * per_sm;
    long long chunks = (slots + (long long)gx * gy - 1) / ((long long)gx * gy);
    if (chunks < 1) chunks = 1;
    long long max_chunks = (nz + 3) / 4;
    if (max_chunks < 1) max_chunks = 1;
    if (chunks > max_chunks) chunks = max_chunks;
    p.zlen = (int)((nz + chunks - 1) / chunks);
    p.grid = dim3(gx, gy, (nz + p.zlen - 1) / p.zlen);
    return p;
  }
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
  if (p.queue) return launch_q_any(b, p, s);
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
