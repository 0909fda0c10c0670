// The mask-and-fill completion of the intensity correction (sm_103a):
// Eqs. (7)-(10), Sec. 2.3 and Algorithm A1 step 2.
//
//  fill pass     one Jacobi pass of Eqs. (8)-(10) over the voxels without a, b:
//                each averages the a, b of the neighbours in the box T that
//                were known before the pass, weighted by
//                exp(-(I_s(i) - I_s(x))^2 / h^2) with the exponent capped at 80
//                (reading R20); a filled voxel gets stamp = pass and
//                d = a I_s + b - m.  A voxel is filled in the first pass after
//                one of its box neighbours is known, so the voxels a pass fills
//                (its front) are the box dilation of the known set less that
//                set.  Bit masks of the known voxels (k_fill_pack before pass 1)
//                are dilated once per pass, the front is listed in voxel order
//                (count, scan, list), and k_fill_pass sums each listed voxel's
//                known neighbours, found from the mask bits: only the front is
//                visited, with the sums a pass over every unknown voxel would
//                form.  A pass returns at once when nothing is masked or the
//                previous pass filled nothing (reading R19).
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

// Bit masks of the known voxels, one 32-bit word per 32 voxels of a row (bit i of
// word w of row (y, z) is voxel x = 32 w + i; bits past nx stay zero).  The
// voxels known before pass p + 1 are the box-T dilation of those known before
// pass p: a voxel is filled in the first pass after a box neighbour is known
// (every weight of Eq. 10 is at least exp(-80) > 0), so the masks follow from
// the mask pass's stamps by dilations alone, and pass p tries exactly the
// voxels it fills.

// K_1: the voxels with xi = 0 (stamp 0).  One warp per word.
__global__ void k_fill_pack(const int* __restrict__ stamp, unsigned* __restrict__ k, int nx, int nwx, long long words) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long w = t >> 5;
  if (w >= words) return;                                  // whole warps leave together
  const int lane = threadIdx.x & 31;
  const long long row = w / nwx;
  const int x = (int)(w - row * nwx) * 32 + lane;
  const bool known = x < nx && stamp[row * nx + x] == 0;
  const unsigned bits = __ballot_sync(0xffffffffu, known);
  if (lane == 0) k[w] = bits;
}

// Dilation word i of K_{p+1}: K_p dilated by the box T, clipped to the volume.
__device__ __forceinline__ unsigned dilate_word(const FillArgs& f, const unsigned* kin, long long i,
                                                unsigned tail) {
  const int nwx = f.nwx, ny = f.ny, nz = f.nz;
  const int w = (int)(i % nwx);
  const long long row = i / nwx;
  const int y = (int)(row % ny), z = (int)(row / ny);
  // union over the box's rows of words w - 1, w, w + 1; the x dilation is
  // applied once to the union (shifts distribute over OR)
  unsigned uc = 0u, ul = 0u, uh = 0u;
  for (int zz = max(0, z - f.tz); zz <= min(nz - 1, z + f.tz); ++zz)
    for (int yy = max(0, y - f.ty); yy <= min(ny - 1, y + f.ty); ++yy) {
      const unsigned* r = kin + ((long long)zz * ny + yy) * nwx;
      uc |= r[w];
      if (w > 0) ul |= r[w - 1];
      if (w + 1 < nwx) uh |= r[w + 1];
    }
  unsigned acc = uc;
  for (int d = 1; d <= f.tx; ++d) acc |= (uc << d) | (ul >> (32 - d)) | (uc >> d) | (uh << (32 - d));
  return w == nwx - 1 ? (acc & tail) : acc;
}

// The pass's front F_p = K_{p+1} minus K_p, listed in voxel order: (1) dilation
// and front counts per block of kFrontWords words, (2) one CTA scans the block
// counts, (3) each block lists its front voxels from its offset.
constexpr int kFrontWords = 256;
constexpr int kScanThreads = 1024;

// The pass a kernel works on and its masks: from the arguments, or (device-driven)
// from the pass counter, which the scan kernel has already advanced for the
// list and fill kernels (behind = 1).
struct PassSel {
  int p;
  const unsigned* kin;
  unsigned* kout;
};

__device__ __forceinline__ PassSel pass_sel(const FillArgs& f, int behind) {
  if (f.next == nullptr) return {f.pass, f.kin, f.kout};
  const int p = *(volatile const int*)f.next - behind;
  return {p, f.kbits + ((p - 1) & 1) * f.kwords, f.kbits + (p & 1) * f.kwords};
}

// A pass has nothing to do when the level has stopped, the previous pass filled
// nothing, or the cap is passed (a loop body's later passes after the last one).
__device__ __forceinline__ bool pass_idle(const FillArgs& f, int p) {
  return p > f.passes || (f.stop != nullptr && *(volatile const int*)f.stop != 0) || f.cnt[p - 1] == 0;
}

__device__ __forceinline__ int block_exclusive_scan(int v, int* red, int& total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int incl = v;
  for (int off = 1; off < 32; off <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += t;
  }
  if (lane == 31) red[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int s = lane < nw ? red[lane] : 0;
    for (int off = 1; off < 32; off <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, s, off);
      if (lane >= off) s += t;
    }
    if (lane < nw) red[lane] = s;                          // inclusive warp totals
  }
  __syncthreads();
  total = red[nw - 1];
  const int before = wid > 0 ? red[wid - 1] : 0;
  __syncthreads();                                         // red is reused by the caller
  return before + incl - v;
}

__global__ void __launch_bounds__(kFrontWords) k_fill_front_count(FillArgs f) {
  const PassSel P = pass_sel(f, 0);
  if (pass_idle(f, P.p)) return;
  __shared__ int red[32];
  const long long words = (long long)f.nwx * f.ny * f.nz;
  const long long i = (long long)blockIdx.x * kFrontWords + threadIdx.x;
  const unsigned tail = (f.nx & 31) ? (1u << (f.nx & 31)) - 1u : 0xffffffffu;
  int c = 0;
  if (i < words) {
    const unsigned k = dilate_word(f, P.kin, i, tail);
    P.kout[i] = k;
    c = __popc(k & ~P.kin[i]);
  }
  int total = 0;
  block_exclusive_scan(c, red, total);
  if (threadIdx.x == 0) f.boff[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_fill_front_scan(FillArgs f, int nblocks) {
  const PassSel P = pass_sel(f, 0);
  const bool idle = pass_idle(f, P.p);       // uniform: *next changes only below
  __shared__ int red[32];
  int carry = 0;
  if (!idle) {
    for (int base = 0; base < nblocks; base += kScanThreads) {
      const int j = base + threadIdx.x;
      const int v = j < nblocks ? f.boff[j] : 0;
      int total = 0;
      const int ex = block_exclusive_scan(v, red, total);
      if (j < nblocks) f.boff[j] = carry + ex;
      carry += total;
    }
  }
  __syncthreads();                           // every thread has read *next
  if (threadIdx.x == 0) {
    if (!idle) f.nfront[0] = carry;
    if (f.next != nullptr) *f.next = P.p + 1;
    // pass p fills exactly its front: pass p + 1 has work only after a non-empty one
    if (f.use_cond) cudaGraphSetConditional(f.cond, (!idle && carry > 0 && P.p < f.passes) ? 1u : 0u);
  }
}

__global__ void k_fill_loop_start(FillArgs f) {
  *f.next = 1;
  const bool stopped = f.stop != nullptr && *(volatile const int*)f.stop != 0;
  if (f.use_cond) cudaGraphSetConditional(f.cond, (!stopped && f.cnt[0] > 0 && f.passes > 0) ? 1u : 0u);
}

__global__ void __launch_bounds__(kFrontWords) k_fill_front_list(FillArgs f) {
  const PassSel P = pass_sel(f, 1);
  if (pass_idle(f, P.p)) return;
  __shared__ int red[32];
  const long long words = (long long)f.nwx * f.ny * f.nz;
  const long long i = (long long)blockIdx.x * kFrontWords + threadIdx.x;
  unsigned b = 0u;
  if (i < words) b = P.kout[i] & ~P.kin[i];
  int total = 0;
  int pos = f.boff[blockIdx.x] + block_exclusive_scan(__popc(b), red, total);
  if (b) {
    const long long row = i / f.nwx;
    const int x0 = (int)(i - row * f.nwx) * 32;
    const long long g0 = row * f.nx + x0;
    while (b) {
      const int j = __ffs(b) - 1;
      b &= b - 1u;
      f.list[pos++] = (int)(g0 + j);
    }
  }
}

// Eqs. (8)-(10) for the listed front voxels, summing the neighbours known before
// the pass (the set bits of K_p in the voxel's box, rows in z, y order and each
// row in increasing x).  A row's entries are all loaded (independent loads in
// flight) and the unknown ones enter with weight 0, which leaves every sum
// unchanged: the working set holds finite values everywhere.
__global__ void __launch_bounds__(kFillThreads) k_fill_pass(FillArgs f) {
  const PassSel P = pass_sel(f, 1);
  if (pass_idle(f, P.p)) return;
  const int n = f.nfront[0];
  const int nx = f.nx, ny = f.ny, nz = f.nz, nwx = f.nwx;
  const size_t plane = (size_t)nx * ny;
  int nfilled = 0;
  for (int k = blockIdx.x * kFillThreads + threadIdx.x; k < n; k += gridDim.x * kFillThreads) {
    const size_t g = (size_t)f.list[k];
    const int z = (int)(g / plane);
    const int rem = (int)(g - (size_t)z * plane);
    const int y = rem / nx, x = rem - y * nx;
    const float isx = f.isab[g].x;
    float num_a = 0.0f, num_b = 0.0f, den = 0.0f;
    const int x_lo = max(0, x - f.tx), x_hi = min(nx - 1, x + f.tx);
    const int w0 = x_lo >> 5, w1 = x_hi >> 5, sh = x_lo & 31;
    const int xn = x_hi - x_lo + 1;
    const unsigned long long span = (1ull << xn) - 1ull;
    for (int zz = max(0, z - f.tz); zz <= min(nz - 1, z + f.tz); ++zz)
      for (int yy = max(0, y - f.ty); yy <= min(ny - 1, y + f.ty); ++yy) {
        const size_t rw = ((size_t)zz * ny + yy) * nwx;
        unsigned long long bits = P.kin[rw + w0];
        if (w1 != w0) bits |= (unsigned long long)P.kin[rw + w1] << 32;
        bits = (bits >> sh) & span;
        const size_t row = (size_t)zz * plane + (size_t)yy * nx + x_lo;
        while (bits) {
          const int j = __ffsll((long long)bits) - 1;
          bits &= bits - 1ull;
          const float4 q = f.isab[row + j];              // (I_s, a, b) of a known neighbour
          const float e = (q.x - isx) * f.inv_h;
          const float wt = expf(-fminf(e * e, 80.0f));    // Eq. (10), exponent capped
          num_a = fmaf(wt, q.y, num_a);
          num_b = fmaf(wt, q.z, num_b);
          den += wt;
        }
      }
    if (den > 0.0f) {
      const float av = num_a / den, bv = num_b / den;     // Eqs. (8), (9)
      f.isab[g] = make_float4(isx, av, bv, 0.0f);
      f.d[g] = fmaf(av, isx, bv) - __ldg(f.m + g);        // d = I'_s - m
      f.stamp[g] = P.p;
      ++nfilled;
    }
  }
  for (int off = 16; off > 0; off >>= 1) nfilled += __shfl_down_sync(0xffffffffu, nfilled, off);
  if ((threadIdx.x & 31) == 0 && nfilled) atomicAdd(&f.cnt[P.p], nfilled);
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
    // grad I'_s = grad d + grad m
    const Dr dr = demons_dr(dp[0], sx, dp[rx] - dp[lx], mp[rx] - mp[lx], sy, dp[ry] - dp[ly], mp[ry] - mp[ly], sz,
                            dp[rz] - dp[lz], mp[rz] - mp[lz], f.force_mode == DISC_FORCE_DOUBLE);
    const float drx = dr.x, dry = dr.y, drz = dr.z;
    const float rxv = __ldg(f.r + g), ryv = __ldg(f.r + (size_t)N + g), rzv = __ldg(f.r + 2 * (size_t)N + g);
    const float keep = f.u_is_dr ? 0.0f : 1.0f;   // u = r + dr, or dr alone
    f.u[g] = fmaf(keep, rxv, drx);
    f.u[(size_t)N + g] = fmaf(keep, ryv, dry);
    f.u[2 * (size_t)N + g] = fmaf(keep, rzv, drz);
    const bool nin = f.norm_hi <= f.norm_lo || (z >= f.norm_lo && z < f.norm_hi);   // the plane enters the norm sums
    acc0 += nin ? norm3(drx, dry, drz) : 0.0f;
    acc1 += nin ? norm3(rxv, ryv, rzv) : 0.0f;
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

// Voxels the fill left: the masked ones less those the passes filled.
__global__ void k_fill_remaining(const int* cnt, int passes, int* out) {
  int left = cnt[0];
  for (int p = 1; p <= passes; ++p) left -= cnt[p];
  *out = left;
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

int fill_words(int nx, int ny, int nz) { return ((nx + 31) / 32) * ny * nz; }

cudaError_t launch_fill_pack(const int* stamp, unsigned* k, int nx, int ny, int nz, cudaStream_t s) {
  const int nwx = (nx + 31) / 32;
  const long long words = (long long)nwx * ny * nz;
  const long long blocks = (words * 32 + 255) / 256;
  if (blocks < 1 || blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  k_fill_pack<<<(int)blocks, 256, 0, s>>>(stamp, k, nx, nwx, words);
  return cudaGetLastError();
}

int fill_front_blocks(int nx, int ny, int nz) {
  return (fill_words(nx, ny, nz) + kFrontWords - 1) / kFrontWords;
}

__global__ void k_unpack_ab(const float4* __restrict__ isab, float* __restrict__ a, float* __restrict__ b,
                            int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float4 q = isab[i];
    a[i] = q.y;
    b[i] = q.z;
  }
}

// Sums of a and b (Eqs. 5-6, after the fill) over the voxels whose stamp is at
// least 0 (known or filled), and their count, into out[0..2] (one CTA, fixed
// order): the averages of Sec. 3.4.
__global__ void k_ab_sums(const float4* __restrict__ isab, const int* __restrict__ stamp, long long n,
                          double* out) {
  __shared__ double sh[3][8];
  double sa = 0.0, sb = 0.0, c = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    if (stamp[i] >= 0) {
      const float4 v = isab[i];
      sa += (double)v.y;
      sb += (double)v.z;
      c += 1.0;
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    sa += __shfl_down_sync(0xffffffffu, sa, off);
    sb += __shfl_down_sync(0xffffffffu, sb, off);
    c += __shfl_down_sync(0xffffffffu, c, off);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    sh[0][w] = sa;
    sh[1][w] = sb;
    sh[2][w] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < (int)(blockDim.x / 32); ++k)
      for (int j = 0; j < 3; ++j) t[j] += sh[j][k];
    out[0] = t[0];
    out[1] = t[1];
    out[2] = t[2];
  }
}

cudaError_t launch_ab_sums(const float4* isab, const int* stamp, int64_t n, double* out, cudaStream_t s) {
  k_ab_sums<<<1, 256, 0, s>>>(isab, stamp, (long long)n, out);
  return cudaGetLastError();
}

cudaError_t launch_unpack_ab(const float4* isab, float* a, float* b, int64_t n, cudaStream_t s) {
  long long blocks = (n + 255) / 256;
  if (blocks > 148 * 8) blocks = 148 * 8;
  if (blocks < 1) blocks = 1;
  k_unpack_ab<<<(int)blocks, 256, 0, s>>>(isab, a, b, n);
  return cudaGetLastError();
}

cudaError_t launch_fill_pass(const FillArgs& f, cudaStream_t s) {
  const int nb = fill_front_blocks(f.nx, f.ny, f.nz);
  k_fill_front_count<<<nb, kFrontWords, 0, s>>>(f);
  k_fill_front_scan<<<1, kScanThreads, 0, s>>>(f, nb);
  k_fill_front_list<<<nb, kFrontWords, 0, s>>>(f);
  const long long n = (long long)f.nx * f.ny * f.nz;
  long long blocks = (n + kFillThreads - 1) / kFillThreads;
  if (blocks > 148 * 16) blocks = 148 * 16;
  if (blocks < 1) blocks = 1;
  k_fill_pass<<<(int)blocks, kFillThreads, 0, s>>>(f);
  return cudaGetLastError();
}

cudaError_t launch_fill_loop_start(const FillArgs& f, cudaStream_t s) {
  k_fill_loop_start<<<1, 1, 0, s>>>(f);
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
