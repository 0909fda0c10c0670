// Gaussian regularisation of the displacement field (Algorithm A1 step 6;
// Sec. 2.3 kernel 2), sm_103a.
//
// r = G_sigma * u for each of the three field components, separable: taps
// w_i proportional to exp(-i^2 / 2 sigma^2), |i| <= R, and on each axis the
// weights are renormalised over the taps that fall inside the volume.
//
// Radii 1..8 take the split form below (a z pass, then an xy pass).  The
// generic kernel, for any other case: a CTA owns a TX x TY column tile and
// marches over a chunk of z planes.  Each plane of u (3 components, tile plus R
// halo) is staged in shared memory, filtered along x and then y, and the
// xy-filtered plane is kept in a ring of 2R+1 planes from which the z filter
// emits the output plane R behind.

#include <cmath>

#include "internal.cuh"
#include "warp_dev.cuh"

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
        const float nrm = a.box_sum ? 1.0f : tap_norm(w, R, gx, nx);
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
        const float nrm = a.box_sum ? 1.0f : tap_norm(w, R, gy, ny);
        slot[e] = nrm == 1.0f ? acc : acc / nrm;
      }
      __syncthreads();
    }
    // z filter for the plane R behind
    const int zo = zi - R;
    if (zo >= z0 && zo < z1) {
      const float nrm = a.box_sum ? 1.0f : tap_norm(w, R, zo, nz);
      const int klo = max(-R, -zo), khi = min(R, nz - 1 - zo);
      for (int e = tid; e < 3 * OP; e += kThreads) {
        const int c = e / OP, rem = e - c * OP;
        const int oy = rem / kGX, ox = rem - oy * kGX;
        const int gx = x0 + ox, gy = y0 + oy;
        if (gx >= nx || gy >= ny) continue;
        float acc = 0.0f;
        for (int k = klo; k <= khi; ++k) acc = fmaf(w[k + R], ring[((zo + k) % KZ) * 3 * OP + e], acc);
        const size_t o = c * N + vix(gx, gy, zo, nx, ny);
        const float v = nrm == 1.0f ? acc : acc / nrm;
        a.r[o] = a.add ? a.add[o] + v : v;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Split form for radius R = 1..8 (compile time), two streaming kernels:
//  k_gauss_z: one thread per (x, y) column and z chunk filters u along z with
//    a queue of 2R+1 pending output planes in registers (slots made static by
//    unrolling the plane loop by 2R+1) and writes t = G_z * u;
//  k_gauss_xy: one CTA per 32 x 32 tile of one plane filters t along x and
//    then y in shared memory, writes r (or adds to it), and optionally
//    evaluates the warped moving image m = I_m(x + r(x)) for the next
//    iteration while r is still in registers (Algorithm A1: "update the
//    moving image").
// The x and y field components are processed as float2 pairs (packed FFMA2),
// the z component as a scalar.
// ---------------------------------------------------------------------------
constexpr int kSX = 32;        // xy tile
constexpr int kSY = 32;
constexpr int kZThreads = 128; // z kernel: a CTA is kZX columns along x by kZY rows
constexpr int kZX = 32, kZY = kZThreads / kZX;
constexpr int kZCtasPerSM = 4;  // z kernel CTAs resident per SM (its launch bound)
constexpr int kBX = 4;         // x outputs per x-filter task
constexpr int kBY = 4;         // y outputs per thread in the y filter

template <int R>
struct XYLayout {
  static constexpr int IX = kSX + 2 * R;
  static constexpr int IY = kSY + 2 * R;
  // Row strides of the staged plane.  An x-filter task reads its window of
  // kBX + 2R inputs as 16-byte vectors; the 8 lanes of a quarter warp read 8
  // consecutive rows, which fall on distinct banks when a row is 4 mod 8 words
  // long (and every row starts on a 16-byte boundary).
  static constexpr int NV2 = (kBX + 2 * R) / 2;                  // float4 loads of (ux, uy) pairs
  static constexpr int NVZ = (kBX + 2 * R + 3) / 4;              // float4 loads of uz
  static constexpr int IXP = IX + ((2 - IX % 4) + 4) % 4;        // float2 stride: IXP = 2 mod 4
  static constexpr int IXPZ0 = kSX - kBX + 4 * NVZ;              // floats a task may read in a row
  static constexpr int IXPZ = IXPZ0 + ((4 - IXPZ0 % 8) + 8) % 8; // float stride: 4 mod 8
  static_assert((kBX + 2 * R) % 2 == 0 && IXP >= IX && IXPZ >= IX, "staged row strides");
  static constexpr int NXT = IY * (kSX / kBX);         // x-filter tasks (row, x quad)
  static constexpr size_t o_in2 = 0;                   // float2 [IY][IXP]  (ux, uy)
  static constexpr size_t o_inz = o_in2 + 8 * (size_t)IY * IXP;   // float [IY][IXPZ]
  static constexpr int XP = kSX + 1;                   // row stride of the x-filtered planes (odd)
  static constexpr size_t o_x2 = o_inz + 4 * (size_t)IY * IXPZ;   // float2 [IY][XP]
  static constexpr size_t o_xz = o_x2 + 8 * (size_t)IY * XP;      // float [IY][XP]
  static constexpr size_t bytes = o_xz + 4 * (size_t)IY * XP;
};

// The xy pass is the last of the two passes: it writes r (r = add + G u when
// a.add is set, in place) and, with WARP, m = I_m(x + r(x)) for the next
// iteration while r is in registers (WARP 1).  The warp's sample indices are
// 32-bit: contexts hold fewer than 2^31 / 3 voxels per level (disc_set_images),
// and the launches refuse a larger volume.
template <int R, int WARP = 0>
__device__ __forceinline__ void gauss_xy_body(const GaussArgs& a, int bx, int by, int bz) {
  using X = XYLayout<R>;
  if (a.stop != nullptr && *(volatile const int*)a.stop != 0) return;
  extern __shared__ __align__(16) unsigned char smem[];
  float2* in2 = reinterpret_cast<float2*>(smem + X::o_in2);
  float* inz = reinterpret_cast<float*>(smem + X::o_inz);
  float2* x2 = reinterpret_cast<float2*>(smem + X::o_x2);
  float* xz = reinterpret_cast<float*>(smem + X::o_xz);
  __shared__ float nrm_x[kSX], nrm_y[kSY];
  const int tid = threadIdx.x;
  const int nx = a.nx, ny = a.ny;
  const size_t plane = (size_t)nx * ny;
  const size_t N = plane * a.nz;
  const int x0 = bx * kSX, y0 = by * kSY, z = bz;
  float w[2 * R + 1];
#pragma unroll
  for (int k = 0; k <= 2 * R; ++k) w[k] = a.w[k];
  const bool border = !a.box_sum && (x0 - R < 0 || x0 + kSX + R > nx || y0 - R < 0 || y0 + kSY + R > ny);
  if (border) {
    if (tid < kSX) nrm_x[tid] = tap_norm(a.w, R, x0 + tid, nx);
    if (tid >= 64 && tid < 64 + kSY) nrm_y[tid - 64] = tap_norm(a.w, R, y0 + tid - 64, ny);
  }
  // stage the plane with its halo (zeros outside the volume): all loads first
  constexpr int NL = (X::IY * X::IX + kThreads - 1) / kThreads;
  const float* ux = a.u + (size_t)z * plane;
  float vx[NL], vy[NL], vz[NL];
#pragma unroll
  for (int k = 0; k < NL; ++k) {
    const int e = tid + k * kThreads;
    const int iy = e / X::IX, ix = e - iy * X::IX;
    const int gx = x0 - R + ix, gy = y0 - R + iy;
    const bool ok = e < X::IY * X::IX && gx >= 0 && gx < nx && gy >= 0 && gy < ny;
    const size_t g = ok ? (size_t)gy * nx + gx : 0;
    vx[k] = ok ? ldg_at(ux + g, a.u, 3LL * N) : 0.0f;
    vy[k] = ok ? ldg_at(ux + N + g, a.u, 3LL * N) : 0.0f;
    vz[k] = ok ? ldg_at(ux + 2 * N + g, a.u, 3LL * N) : 0.0f;
  }
#pragma unroll
  for (int k = 0; k < NL; ++k) {
    const int e = tid + k * kThreads;
    if (e < X::IY * X::IX) {
      const int iy = e / X::IX, ix = e - iy * X::IX;
      in2[iy * X::IXP + ix] = make_float2(vx[k], vy[k]);
      inz[iy * X::IXPZ + ix] = vz[k];
    }
  }
  __syncthreads();
  // x filter: each task computes kBX adjacent outputs of one row from a window
  // of kBX + 2R inputs held in registers
  for (int t = tid; t < X::NXT; t += kThreads) {
    // consecutive tasks take consecutive rows: the odd row strides then spread a
    // warp's loads and stores over all shared-memory banks
    const int j = t / X::IY, iy = t - j * X::IY;
    const float4* r2 = reinterpret_cast<const float4*>(in2 + iy * X::IXP + kBX * j);
    const float4* rz = reinterpret_cast<const float4*>(inz + iy * X::IXPZ + kBX * j);
    float2 w2[2 * X::NV2];
    float wz[4 * X::NVZ];
#pragma unroll
    for (int g = 0; g < X::NV2; ++g) {
      const float4 q = r2[g];
      w2[2 * g] = make_float2(q.x, q.y);
      w2[2 * g + 1] = make_float2(q.z, q.w);
    }
#pragma unroll
    for (int g = 0; g < X::NVZ; ++g) {
      const float4 q = rz[g];
      wz[4 * g] = q.x;
      wz[4 * g + 1] = q.y;
      wz[4 * g + 2] = q.z;
      wz[4 * g + 3] = q.w;
    }
    float2 acc[kBX];
    float accz[kBX];
#pragma unroll
    for (int b = 0; b < kBX; ++b) {
      acc[b] = make_float2(0.0f, 0.0f);
      accz[b] = 0.0f;
    }
#pragma unroll
    for (int i = 0; i < kBX + 2 * R; ++i) {
      const float2 v = w2[i];
      const float vzz = wz[i];
#pragma unroll
      for (int b = 0; b < kBX; ++b) {
        const int k = i - b;                  // tap index of input i for output b
        if (k >= 0 && k <= 2 * R) {
          acc[b] = __ffma2_rn(make_float2(w[k], w[k]), v, acc[b]);
          accz[b] = fmaf(w[k], vzz, accz[b]);
        }
      }
    }
#pragma unroll
    for (int b = 0; b < kBX; ++b) {
      if (border) {
        const float n = nrm_x[kBX * j + b];
        if (n != 1.0f) {
          acc[b].x = acc[b].x / n;
          acc[b].y = acc[b].y / n;
          accz[b] = accz[b] / n;
        }
      }
      x2[iy * X::XP + kBX * j + b] = acc[b];
      xz[iy * X::XP + kBX * j + b] = accz[b];
    }
  }
  __syncthreads();
  // y filter: each thread computes kBY adjacent rows of one column
  {
    const int ox = tid & (kSX - 1), jy = tid >> 5;      // 32 columns x 8 row groups
    const int gx = x0 + ox;
    const float2* c2 = x2 + kBY * jy * X::XP + ox;
    const float* cz = xz + kBY * jy * X::XP + ox;
    float2 acc[kBY];
    float accz[kBY];
#pragma unroll
    for (int b = 0; b < kBY; ++b) {
      acc[b] = make_float2(0.0f, 0.0f);
      accz[b] = 0.0f;
    }
#pragma unroll
    for (int i = 0; i < kBY + 2 * R; ++i) {
      const float2 v = c2[i * X::XP];
      const float vzz = cz[i * X::XP];
#pragma unroll
      for (int b = 0; b < kBY; ++b) {
        const int k = i - b;
        if (k >= 0 && k <= 2 * R) {
          acc[b] = __ffma2_rn(make_float2(w[k], w[k]), v, acc[b]);
          accz[b] = fmaf(w[k], vzz, accz[b]);
        }
      }
    }
    if (gx < nx) {
      float* t = a.r + (size_t)z * plane;
#pragma unroll
      for (int b = 0; b < kBY; ++b) {
        const int gy = y0 + kBY * jy + b;
        if (gy >= ny) break;
        if (border) {
          const float n = nrm_y[kBY * jy + b];
          if (n != 1.0f) {
            acc[b].x = acc[b].x / n;
            acc[b].y = acc[b].y / n;
            accz[b] = accz[b] / n;
          }
        }
        const size_t g = (size_t)gy * nx + gx;
        if (a.add) {                          // r = r_prev + G * dr (in place: same element)
          const float* ap = a.add + (t - a.r) + g;
          acc[b].x += DISC_IN(ap - a.add, 3LL * N) ? ap[0] : 0.0f;
          acc[b].y += DISC_IN(ap + N - a.add, 3LL * N) ? ap[N] : 0.0f;
          accz[b] += DISC_IN(ap + 2 * N - a.add, 3LL * N) ? ap[2 * N] : 0.0f;
        }
        st_at(t + g, a.r, 3LL * N, acc[b].x);
        st_at(t + N + g, a.r, 3LL * N, acc[b].y);
        st_at(t + 2 * N + g, a.r, 3LL * N, accz[b]);
        if (WARP != 0)
          st_at(a.m + (size_t)z * plane + g, a.m, (long long)N,
                warp_at32(a.Im, gx, gy, z, acc[b].x, acc[b].y, accz[b], nx, ny, a.nz));
      }
    }
  }
}

template <int R, int WARP>
__global__ void __launch_bounds__(kThreads) k_gauss_xy(GaussArgs a) {
  pdl_wait();
  pdl_release();
  gauss_xy_body<R, WARP>(a, blockIdx.x, blockIdx.y, blockIdx.z);
}

// Work item i of a batched launch -> (volume p, CTA coordinates in p's grid).
__device__ __forceinline__ int batch_find(const int* offset, int count, int i) {
  int p = 0;
  while (p + 1 < count && offset[p + 1] <= i) ++p;
  return p;
}

template <int R, int WARP>
__global__ void __launch_bounds__(kThreads) k_gauss_xy_batch(const __grid_constant__ GaussBatch bt) {
  pdl_wait();
  pdl_release();
  const int i = blockIdx.x;
  const int p = batch_find(bt.offset, bt.count, i);
  const int j = i - bt.offset[p];
  const dim3 g = bt.grid[p];
  gauss_xy_body<R, WARP>(bt.args[p], j % g.x, (j / g.x) % g.y, j / (g.x * g.y));
}

// z pass with a register queue (the first of the two passes: u -> t).
template <int R>
__device__ __forceinline__ void gauss_z_body(const GaussArgs& a, int bx, int by, int bz) {
  constexpr int KZ = 2 * R + 1;
  if (a.stop != nullptr && *(volatile const int*)a.stop != 0) return;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int x = bx * kZX + threadIdx.x % kZX, y = by * kZY + threadIdx.x / kZX;
  if (x >= nx || y >= ny) return;
  const size_t plane = (size_t)nx * ny;
  const size_t N = plane * nz;
  const int z0 = bz * a.zlen;
  const int z1 = min(nz, z0 + a.zlen);
  float w[KZ];
#pragma unroll
  for (int k = 0; k < KZ; ++k) w[k] = a.w[k];
  const size_t col = (size_t)y * nx + x;
  const float* t = a.u + col;       // the input column, [3][N]
  float2 q2[KZ];                    // pending outputs, (x, y) components
  float qz[KZ];
#pragma unroll
  for (int k = 0; k < KZ; ++k) {
    q2[k] = make_float2(0.0f, 0.0f);
    qz[k] = 0.0f;
  }
  const int zs = max(0, z0 - R);
  const int ze = z1 - 1 + R;
  const int zb0 = zs - (zs % KZ);
  const float* tb = t + (size_t)zb0 * plane;  // plane zb of the block, advanced by KZ planes
  float* rb = a.r + col + (size_t)(zb0 - R) * plane;   // output plane zb - R
  const size_t step = (size_t)KZ * plane;
  for (int zb = zb0; zb <= ze; zb += KZ, tb += step, rb += step) {
    // issue the loads of the whole block of 2R+1 planes first (memory-level parallelism)
    float2 v2[KZ];
    float vz[KZ];
#pragma unroll
    for (int j = 0; j < KZ; ++j) {
      const int zi = zb + j;
      const bool ok = zi >= zs && zi <= ze && zi < nz;
      const float* tp = tb + (size_t)j * plane;
      v2[j] = ok ? make_float2(ldg_at(tp, a.u, 3LL * N), ldg_at(tp + N, a.u, 3LL * N)) : make_float2(0.0f, 0.0f);
      vz[j] = ok ? ldg_at(tp + 2 * N, a.u, 3LL * N) : 0.0f;
    }
#pragma unroll
    for (int j = 0; j < KZ; ++j) {
      const int zi = zb + j;                  // zi mod KZ == j
      if (zi < zs || zi > ze) continue;
      // plane zi feeds output plane zi - k with tap w[R + k] (zero planes add nothing)
#pragma unroll
      for (int k = -R; k <= R; ++k) {
        const int slot = ((j - k) % KZ + KZ) % KZ;
        q2[slot] = __ffma2_rn(make_float2(w[R + k], w[R + k]), v2[j], q2[slot]);
        qz[slot] = fmaf(w[R + k], vz[j], qz[slot]);
      }
      const int zo = zi - R;
      const int so = ((j - R) % KZ + KZ) % KZ;
      if (zo >= z0 && zo < z1) {
        float2 o2 = q2[so];
        float oz = qz[so];
        const float nrm = a.box_sum ? 1.0f : tap_norm(a.w, R, zo, nz);
        if (nrm != 1.0f) {
          o2.x = o2.x / nrm;
          o2.y = o2.y / nrm;
          oz = oz / nrm;
        }
        float* rp = rb + (size_t)j * plane;
        st_at(rp, a.r, 3LL * N, o2.x);
        st_at(rp + N, a.r, 3LL * N, o2.y);
        st_at(rp + 2 * N, a.r, 3LL * N, oz);
      }
      q2[so] = make_float2(0.0f, 0.0f);
      qz[so] = 0.0f;
    }
  }
}

template <int R>
__global__ void __launch_bounds__(kZThreads, kZCtasPerSM) k_gauss_z(GaussArgs a) {
  pdl_wait();
  pdl_release();
  gauss_z_body<R>(a, blockIdx.x, blockIdx.y, blockIdx.z);
}

template <int R>
__global__ void __launch_bounds__(kZThreads, kZCtasPerSM) k_gauss_z_batch(const __grid_constant__ GaussBatch bt) {
  pdl_wait();
  pdl_release();
  const int i = blockIdx.x;
  const int p = batch_find(bt.offset, bt.count, i);
  const int j = i - bt.offset[p];
  const dim3 g = bt.grid[p];
  gauss_z_body<R>(bt.args[p], j % g.x, (j / g.x) % g.y, j / (g.x * g.y));
}

// The fused warp's 32-bit sample indices need every index of I_m to fit.
inline bool warp_fits(long long voxels) { return voxels < (1LL << 31); }

template <class K>
cudaError_t set_xy_attrs(K k, size_t bytes) {
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                              (int)cudaSharedmemCarveoutMaxShared);
}

// Batched z pass (u -> t) then batched xy pass (t -> r, with add and warp).
template <int R>
cudaError_t launch_batch_r(const GaussBatch& xy, int xy_total, const GaussBatch& z, int z_total, bool warp,
                           cudaStream_t s) {
  static int set[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!set[dev]) {
    if ((e = set_xy_attrs(k_gauss_xy_batch<R, 0>, XYLayout<R>::bytes)) != cudaSuccess) return e;
    if ((e = set_xy_attrs(k_gauss_xy_batch<R, 1>, XYLayout<R>::bytes)) != cudaSuccess) return e;
    set[dev] = 1;
  }
  if (warp)
    for (int p = 0; p < xy.count; ++p)
      if (!warp_fits((long long)xy.args[p].nx * xy.args[p].ny * xy.args[p].nz)) return cudaErrorInvalidValue;
  if (z_total > 0) e = launch_pdl(k_gauss_z_batch<R>, dim3(z_total), dim3(kZThreads), 0, s, z);
  if (e != cudaSuccess || xy_total <= 0) return e;
  if (!warp) return launch_pdl(k_gauss_xy_batch<R, 0>, dim3(xy_total), dim3(kThreads), XYLayout<R>::bytes, s, xy);
  return launch_pdl(k_gauss_xy_batch<R, 1>, dim3(xy_total), dim3(kThreads), XYLayout<R>::bytes, s, xy);
}

// z pass (u -> t) then xy pass (t -> r = add + G u, and m = I_m(x + r) when a.m
// is set).  The xy pass runs last so that the add and the warp see r in
// registers: it already stages its planes through shared memory, and its tile
// of 32 x 32 voxels keeps the warp's gathers of one plane close together.
template <int R>
cudaError_t launch_split(const GaussArgs& a, const GaussPlan& p, cudaStream_t s) {
  static int set[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!set[dev]) {
    if ((e = set_xy_attrs(k_gauss_xy<R, 0>, XYLayout<R>::bytes)) != cudaSuccess) return e;
    if ((e = set_xy_attrs(k_gauss_xy<R, 1>, XYLayout<R>::bytes)) != cudaSuccess) return e;
    set[dev] = 1;
  }
  if (a.m != nullptr && !warp_fits((long long)a.nx * a.ny * a.nz)) return cudaErrorInvalidValue;
  // z: u -> t
  GaussArgs zz = a;
  zz.r = a.t;
  zz.add = nullptr;
  zz.m = nullptr;
  zz.zlen = p.zlen;
  dim3 gz((a.nx + kZX - 1) / kZX, (a.ny + kZY - 1) / kZY, (a.nz + p.zlen - 1) / p.zlen);
  e = launch_pdl(k_gauss_z<R>, gz, dim3(kZThreads), 0, s, zz);
  if (e != cudaSuccess) return e;
  // xy: t -> r (and m)
  GaussArgs xy = a;
  xy.u = a.t;
  dim3 gxy((a.nx + kSX - 1) / kSX, (a.ny + kSY - 1) / kSY, a.nz);
  if (a.m == nullptr) return launch_pdl(k_gauss_xy<R, 0>, gxy, dim3(kThreads), XYLayout<R>::bytes, s, xy);
  return launch_pdl(k_gauss_xy<R, 1>, gxy, dim3(kThreads), XYLayout<R>::bytes, s, xy);
}

cudaError_t launch_split_any(const GaussArgs& a, const GaussPlan& p, cudaStream_t s) {
  switch (a.R) {
#define QCASE(RR) case RR: return launch_split<RR>(a, p, s);
    QCASE(1) QCASE(2) QCASE(3) QCASE(4) QCASE(5) QCASE(6) QCASE(7) QCASE(8)
#undef QCASE
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace

cudaError_t gauss_launch_batch(const GaussBatch& xy, int xy_total, const GaussBatch& z, int z_total,
                               int R, bool warp, cudaStream_t s) {
  switch (R) {
#define BCASE(RR) case RR: return launch_batch_r<RR>(xy, xy_total, z, z_total, warp, s);
    BCASE(1) BCASE(2) BCASE(3) BCASE(4) BCASE(5) BCASE(6) BCASE(7) BCASE(8)
#undef BCASE
    default: return cudaErrorInvalidValue;
  }
}

void gauss_grids(int nx, int ny, int nz, const GaussPlan& p, dim3* xy, dim3* z) {
  *xy = dim3((nx + kSX - 1) / kSX, (ny + kSY - 1) / kSY, nz);
  *z = dim3((nx + kZX - 1) / kZX, (ny + kZY - 1) / kZY, (nz + p.zlen - 1) / p.zlen);
}

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
  p.queue = R >= 1 && R <= 8 && ny <= 65535 && nz <= 65535;
  if (p.queue) {
    p.smem = 0;
    // z kernel: chunks long enough to amortise the 2R halo planes, enough CTAs
    const long long cols = (long long)((nx + kZX - 1) / kZX) * ((ny + kZY - 1) / kZY);
    long long chunks = (8LL * num_sms + cols - 1) / cols;
    if (chunks < 1) chunks = 1;
    long long max_chunks = (nz + 15) / 16;   // at least 16 planes per chunk
    if (max_chunks < 1) max_chunks = 1;
    if (chunks > max_chunks) chunks = max_chunks;
    // small volumes: as many chunks of at least 4 planes as one wave of resident
    // CTAs holds, when that is more (the march's plane latency, not its 2R halo
    // planes, bounds them)
    long long wave = (long long)kZCtasPerSM * num_sms / cols;
    const long long max_short = (nz + 3) / 4;
    if (wave > max_short) wave = max_short;
    if (chunks < wave) chunks = wave;
    p.zlen = (int)((nz + chunks - 1) / chunks);
    p.grid = dim3(1, 1, 1);
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
  if (p.queue) return launch_split_any(b, p, s);
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
  e = cudaGetLastError();
  // the generic kernel does not fuse the warp of the next iteration
  if (e == cudaSuccess && a.m != nullptr) e = launch_warp(a.Im, a.r, a.m, a.nx, a.ny, a.nz, a.stop, s);
  return e;
}

}  // namespace disc
