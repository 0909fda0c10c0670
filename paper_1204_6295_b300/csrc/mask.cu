// The mask-and-fill completion of the intensity correction (sm_103a):
// Eqs. (7)-(10), Sec. 2.3 and Algorithm A1 step 2.
//
//  k_fill_pass   one Jacobi pass of Eqs. (8)-(10) over the list of voxels still
//                without a, b: each averages the a, b of the neighbours in the
//                box T that were known before the pass (stamp in [0, pass)),
//                weighted by exp(-(I_s(i) - I_s(x))^2 / h^2) with the exponent
//                capped at 80 (reading R20); filled voxels get stamp = pass and
//                d = a I_s + b - m, the others go to the next pass's list.
//                A pass returns at once when no voxel is left or the previous
//                pass filled nothing (reading R19).
//  k_force_dm    the demons force (Eq. 1) and update u = r + dr from d = I'_s - m
//                and m, with the arithmetic of the force stage of the box pass.
//  median        a_m of Sec. 2.3: lower and upper median of the non-negative
//                entries of a by a two-level radix select on the float bits.

#include <cuda_runtime.h>

#include "box_dev.cuh"
#include "internal.cuh"

namespace disc {

namespace {

constexpr int kFillThreads = 128;
constexpr int kForceThreads = 256;

__global__ void __launch_bounds__(kFillThreads) k_fill_pass(FillArgs f) {
  if (f.stop != nullptr && *(volatile const int*)f.stop != 0) return;
  const int n_in = f.cnt[f.pass - 1];
  if (n_in == 0) return;
  if (f.pass >= 2 && n_in == f.cnt[f.pass - 2]) return;   // the last pass filled nothing
  const int nx = f.nx, ny = f.ny, nz = f.nz;
  const size_t plane = (size_t)nx * ny;
  for (int i = blockIdx.x * kFillThreads + threadIdx.x; i < n_in; i += gridDim.x * kFillThreads) {
    const int g = f.list_in[i];
    const int z = (int)(g / plane);
    const int rem = g - (int)((size_t)z * plane);
    const int y = rem / nx, x = rem - y * nx;
    const float isx = __ldg(f.is + g);
    float num_a = 0.0f, num_b = 0.0f, den = 0.0f;
    const int z_lo = max(0, z - f.tz), z_hi = min(nz - 1, z + f.tz);
    const int y_lo = max(0, y - f.ty), y_hi = min(ny - 1, y + f.ty);
    const int x_lo = max(0, x - f.tx), x_hi = min(nx - 1, x + f.tx);
    for (int zz = z_lo; zz <= z_hi; ++zz)
      for (int yy = y_lo; yy <= y_hi; ++yy) {
        const size_t row = (size_t)zz * plane + (size_t)yy * nx;
        for (int xx = x_lo; xx <= x_hi; ++xx) {
          const size_t gi = row + xx;
          const int st = f.stamp[gi];
          if (st < 0 || st >= f.pass) continue;           // known before this pass only
          const float e = (__ldg(f.is + gi) - isx) * f.inv_h;
          const float w = expf(-fminf(e * e, 80.0f));     // Eq. (10), exponent capped
          num_a = fmaf(w, f.a[gi], num_a);
          num_b = fmaf(w, f.b[gi], num_b);
          den += w;
        }
      }
    if (den > 0.0f) {
      const float av = num_a / den, bv = num_b / den;     // Eqs. (8), (9)
      f.a[g] = av;
      f.b[g] = bv;
      f.d[g] = fmaf(av, isx, bv) - __ldg(f.m + g);        // d = I'_s - m
      f.stamp[g] = f.pass;
    } else {
      f.list_out[atomicAdd(&f.cnt[f.pass], 1)] = g;
    }
  }
}

// One-sided differences at the faces as s * (v[+r] - v[-l]), l, r in {0, 1}.
__device__ __forceinline__ void diff_coeffs(int c, int n, int stride, int& lo, int& hi, float& s) {
  lo = c > 0 ? -stride : 0;
  hi = c < n - 1 ? stride : 0;
  s = (lo != 0 && hi != 0) ? 0.5f : ((lo != 0 || hi != 0) ? 1.0f : 0.0f);
}

__global__ void __launch_bounds__(kForceThreads) k_force_dm(ForceArgs f) {
  if (f.stop != nullptr && *(volatile const int*)f.stop != 0) return;
  const int nx = f.nx, ny = f.ny, nz = f.nz;
  const int plane = nx * ny;
  const int N = plane * nz;
  float acc0 = 0.0f, acc1 = 0.0f;
  for (int g = blockIdx.x * kForceThreads + threadIdx.x; g < N; g += gridDim.x * kForceThreads) {
    const int z = g / plane, rem = g - z * plane;
    const int y = rem / nx, x = rem - y * nx;
    int lx, rx, ly, ry, lz, rz;
    float sx, sy, sz;
    diff_coeffs(x, nx, 1, lx, rx, sx);
    diff_coeffs(y, ny, nx, ly, ry, sy);
    diff_coeffs(z, nz, plane, lz, rz, sz);
    const float* dp = f.d + g;
    const float* mp = f.m + g;
    const float d0 = dp[0];
    const float gdx = sx * (dp[rx] - dp[lx]);
    const float gmx = sx * (mp[rx] - mp[lx]);
    const float gdy = sy * (dp[ry] - dp[ly]);
    const float gmy = sy * (mp[ry] - mp[ly]);
    const float gdz = sz * (dp[rz] - dp[lz]);
    const float gmz = sz * (mp[rz] - mp[lz]);
    const float gfx = gdx + gmx, gfy = gdy + gmy, gfz = gdz + gmz;   // grad I'_s = grad d + grad m
    const float diff = d0;
    const float d2 = diff * diff;
    const float den = fmaf(gfx, gfx, fmaf(gfy, gfy, fmaf(gfz, gfz, d2)));
    const float sc = den > 1e-9f ? __fdividef(diff, den) : 0.0f;
    float drx = sc * gfx, dry = sc * gfy, drz = sc * gfz;
    if (f.force_mode == DISC_FORCE_DOUBLE) {
      const float den2 = fmaf(gmx, gmx, fmaf(gmy, gmy, fmaf(gmz, gmz, d2)));
      const float s2 = den2 > 1e-9f ? __fdividef(diff, den2) : 0.0f;
      drx = fmaf(s2, gmx, drx);
      dry = fmaf(s2, gmy, dry);
      drz = fmaf(s2, gmz, drz);
    }
    const float rxv = __ldg(f.r + g), ryv = __ldg(f.r + (size_t)N + g), rzv = __ldg(f.r + 2 * (size_t)N + g);
    const float keep = f.u_is_dr ? 0.0f : 1.0f;   // u = r + dr, or dr alone
    f.u[g] = fmaf(keep, rxv, drx);
    f.u[(size_t)N + g] = fmaf(keep, ryv, dry);
    f.u[2 * (size_t)N + g] = fmaf(keep, rzv, drz);
    acc0 += sqrt_approx(fmaf(drx, drx, fmaf(dry, dry, drz * drz)));
    acc1 += sqrt_approx(fmaf(rxv, rxv, fmaf(ryv, ryv, rzv * rzv)));
  }
  __shared__ float red[2][kForceThreads / 32];
  for (int off = 16; off > 0; off >>= 1) {
    acc0 += __shfl_down_sync(0xffffffffu, acc0, off);
    acc1 += __shfl_down_sync(0xffffffffu, acc1, off);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][wid] = acc0;
    red[1][wid] = acc1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float t0 = 0.0f, t1 = 0.0f;
    for (int w = 0; w < kForceThreads / 32; ++w) {
      t0 += red[0][w];
      t1 += red[1][w];
    }
    f.partials[2 * blockIdx.x] = t0;
    f.partials[2 * blockIdx.x + 1] = t1;
  }
}

// ---- median by radix select ---------------------------------------------------
// work: [0, 65536) histogram, [65536] count of non-negative entries,
// [65537 + 4 j ...] state of selection j (0: lower median, 1: upper median):
//   +0 rank wanted, +1 high 16 bits found, +2 rank inside that bin, +3 result bits.
constexpr int kBins = 65536;
constexpr int kSelThreads = 256;

__global__ void k_count_valid(const float* a, int64_t n, unsigned* work) {
  unsigned c = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    c += __ldg(a + i) >= 0.0f ? 1u : 0u;
  for (int off = 16; off > 0; off >>= 1) c += __shfl_down_sync(0xffffffffu, c, off);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(&work[kBins], c);
}

// level 0: histogram of the high 16 bits; level 1: of the low 16 bits among the
// entries whose high bits equal those found for selection j
__global__ void k_hist(const float* a, int64_t n, unsigned* work, int level, int j) {
  const unsigned hi_sel = level ? work[kBins + 1 + 4 * j + 1] : 0u;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float v = __ldg(a + i);
    if (!(v >= 0.0f)) continue;
    const unsigned bits = __float_as_uint(v);   // non-negative floats order as their bits
    if (level == 0) atomicAdd(&work[bits >> 16], 1u);
    else if ((bits >> 16) == hi_sel) atomicAdd(&work[bits & 0xffffu], 1u);
  }
}

// One block: the bin holding the wanted rank (prefix sums over 256-bin chunks).
__global__ void __launch_bounds__(kSelThreads) k_select(unsigned* work, int level, int j) {
  __shared__ unsigned chunk[kSelThreads];
  unsigned* st = work + kBins + 1 + 4 * j;
  const unsigned nvalid = work[kBins];
  if (level == 0) {
    if (threadIdx.x == 0) st[0] = j == 0 ? (nvalid - 1u) / 2u : nvalid / 2u;
    __syncthreads();
  }
  const unsigned want = level == 0 ? st[0] : st[2];
  unsigned s = 0;
  for (int b = 0; b < kBins / kSelThreads; ++b) s += work[threadIdx.x * (kBins / kSelThreads) + b];
  chunk[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned before = 0;
    int c = 0;
    while (c < kSelThreads - 1 && before + chunk[c] <= want) before += chunk[c++];
    int b = c * (kBins / kSelThreads);
    while (b < kBins - 1 && before + work[b] <= want) before += work[b++];
    if (level == 0) {
      st[1] = (unsigned)b;
      st[2] = want - before;
    } else {
      st[3] = (st[1] << 16) | (unsigned)b;
    }
  }
}

__global__ void k_median_finish(const unsigned* work, double* out) {
  const unsigned n = work[kBins];
  const float lo = __uint_as_float(work[kBins + 1 + 3]), hi = __uint_as_float(work[kBins + 1 + 7]);
  *out = n > 0 ? 0.5 * ((double)lo + (double)hi) : -1.0;
}

// Voxels the fill left: the count of the last pass that ran.
__global__ void k_fill_remaining(const int* cnt, int passes, int* out) {
  int last = cnt[0];
  for (int p = 1; p <= passes; ++p) {
    if (last == 0 || (p >= 2 && cnt[p - 1] == cnt[p - 2])) break;   // this pass returned at once
    last = cnt[p];
  }
  *out = last;
}

__global__ void k_add(const float* __restrict__ a, const float* __restrict__ b, float* out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = a[i] + b[i];
}

}  // namespace

cudaError_t launch_median_finish(const unsigned* work, double* out, cudaStream_t s) {
  k_median_finish<<<1, 1, 0, s>>>(work, out);
  return cudaGetLastError();
}

cudaError_t launch_fill_remaining(const int* cnt, int passes, int* out, cudaStream_t s) {
  k_fill_remaining<<<1, 1, 0, s>>>(cnt, passes, out);
  return cudaGetLastError();
}

cudaError_t launch_add(const float* a, const float* b, float* out, int64_t n, cudaStream_t s) {
  int blocks = (int)((n + 255) / 256);
  if (blocks > 148 * 8) blocks = 148 * 8;
  if (blocks < 1) blocks = 1;
  k_add<<<blocks, 256, 0, s>>>(a, b, out, n);
  return cudaGetLastError();
}

cudaError_t launch_fill_pass(const FillArgs& f, int max_items, cudaStream_t s) {
  int blocks = (max_items + kFillThreads - 1) / kFillThreads;
  if (blocks > 148 * 16) blocks = 148 * 16;
  if (blocks < 1) blocks = 1;
  k_fill_pass<<<blocks, kFillThreads, 0, s>>>(f);
  return cudaGetLastError();
}

int force_blocks(int64_t n, int max_parts) {
  int64_t b = (n + kForceThreads - 1) / kForceThreads;
  if (b > max_parts) b = max_parts;
  if (b < 1) b = 1;
  return (int)b;
}

cudaError_t launch_force_dm(const ForceArgs& f, int blocks, cudaStream_t s) {
  k_force_dm<<<blocks, kForceThreads, 0, s>>>(f);
  return cudaGetLastError();
}

size_t median_work_words() { return kBins + 1 + 8; }

cudaError_t launch_median(const float* a, int64_t n, unsigned* work, cudaStream_t s) {
  int blocks = (int)((n + 255) / 256);
  if (blocks > 148 * 8) blocks = 148 * 8;
  if (blocks < 1) blocks = 1;
  cudaError_t e = cudaMemsetAsync(work, 0, sizeof(unsigned) * median_work_words(), s);
  if (e != cudaSuccess) return e;
  k_count_valid<<<blocks, 256, 0, s>>>(a, n, work);
  for (int j = 0; j < 2 && e == cudaSuccess; ++j) {
    e = cudaMemsetAsync(work, 0, sizeof(unsigned) * kBins, s);
    if (e != cudaSuccess) break;
    k_hist<<<blocks, 256, 0, s>>>(a, n, work, 0, j);
    k_select<<<1, kSelThreads, 0, s>>>(work, 0, j);
    e = cudaMemsetAsync(work, 0, sizeof(unsigned) * kBins, s);
    if (e != cudaSuccess) break;
    k_hist<<<blocks, 256, 0, s>>>(a, n, work, 1, j);
    k_select<<<1, kSelThreads, 0, s>>>(work, 1, j);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace disc
