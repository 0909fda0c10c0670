// Patch-moment kernels of the DISC iteration (sm_103a).
//
// The input plane values v (the warped CT m = I_m(x + r(x)) written by k_warp,
// or the CBCT itself for the static statistics) are read from global memory;
// the tile halo and the planes leaving the z window are re-read from L2 rather
// than kept in shared memory, which keeps a CTA small enough for several to be
// resident per SM.
//
// One CTA owns a TX x TY column tile of output voxels and marches over a chunk
// of z planes.  For every plane it enters it
//   1. quantises v to q = rint(v 2^e) and updates, per column of the tile plus
//      the patch halo, exact integer sliding sums over z of q and q^2;
//   2. forms the x and then the y window sums by sliding windows, giving the
//      patch sums S1 = sum q and S2 = sum q^2 of the truncated patch (Eq. 3);
//   3. turns them into the patch moments E(X), STD(X) (Eq. 3; Appendix A.4)
//      and the moment-matched CBCT (Eqs. 5-6), kept as its deviation from the
//      warped CT, d = I'_s - I_m^(k) = zs STD(M) + (E(M) - m)
//      with zs = (I_s - E(S)) / STD(S) precomputed once per level;
//   4. (iteration mode) from a ring of three d planes and the warped CT, the
//      gradient of I'_s as grad d + grad m (central differences, one-sided at
//      the faces), the demons force of Eq. (1) and u = r + dr (Algorithm A1
//      steps 4 and 5), with per-CTA sums of |dr| and |r| (Sec. 2.3 norm).
//
// I'_s is never formed in absolute terms: near-flat patches, where the force
// is a ratio of two tiny numbers, see f - m and grad f at the precision of
// their own magnitude rather than that of a ~1000 HU image value.
//
// Integer sums make the statistics exact and independent of tile shape and
// launch order: a constant patch has variance exactly 0, and repeated or
// batched launches give bit-identical results.

#include <cuda_runtime.h>

#include "box_dev.cuh"
#include "internal.cuh"

namespace disc {

struct BoxLayout {
  int WX, WY, FX, FY, PZ, WN, FN, XN;
  int nsegx, segx, nsegy, segy;
  size_t o_s2z, o_xb1, o_xb2, o_s1z, o_dring, total;
};

// F region: the tile plus a one-voxel ring in iteration mode (the gradient of
// I'_s needs it); W region: F plus the patch half sizes.
__host__ __device__ inline BoxLayout box_layout(int mode, int TX, int TY, int hx, int hy, int hz) {
  BoxLayout L;
  const int ext = (mode == kModeIterate) ? 1 : 0;
  L.FX = TX + 2 * ext;
  L.FY = TY + 2 * ext;
  L.WX = L.FX + 2 * hx;
  L.WY = L.FY + 2 * hy;
  L.PZ = 2 * hz + 1;
  L.WN = L.WX * L.WY;
  L.FN = L.FX * L.FY;
  L.XN = L.FX * L.WY;
  // x sliding: one task per (row, segment); y sliding: one task per (column, segment)
  L.nsegx = kThreads / L.WY;
  if (L.nsegx < 1) L.nsegx = 1;
  if (L.nsegx > L.FX) L.nsegx = L.FX;
  L.segx = (L.FX + L.nsegx - 1) / L.nsegx;
  L.nsegx = (L.FX + L.segx - 1) / L.segx;
  L.nsegy = kThreads / L.FX;
  if (L.nsegy < 1) L.nsegy = 1;
  if (L.nsegy > L.FY) L.nsegy = L.FY;
  L.segy = (L.FY + L.nsegy - 1) / L.nsegy;
  L.nsegy = (L.FY + L.segy - 1) / L.segy;
  size_t o = 0;
  L.o_s2z = o;   o += 8 * (size_t)L.WN;
  L.o_xb1 = o;   o += 8 * (size_t)L.XN;
  L.o_xb2 = o;   o += 8 * (size_t)L.XN;
  L.o_s1z = o;   o += 4 * (size_t)L.WN;
  L.o_dring = o; o += (mode == kModeIterate) ? 4 * 3 * (size_t)L.FN : 0;
  L.total = (o + 15) & ~(size_t)15;
  return L;
}

// Patch moments from exact integer sums of q = rint(v 2^e) over n voxels.
//  dc    = E(X) - v_c = (S1 - n q_c) / (n 2^e): the quantised mean, anchored on
//          the exact centre value (a constant patch gives dc = 0 exactly).
//  sigma = sqrt(Var), Var = (T/n - (e/n)^2) / 2^(2e) with
//          T = sum (q - k)^2 = S2 - 2 k S1 + n k^2, k = round(S1/n), e = S1 - n k,
//          evaluated modulo 2^64 (the true T fits in 63 bits): no precision is
//          lost to the cancellation in E(X^2) - E(X)^2.  sigma = 0 when
//          Var <= var_floor.
__device__ __forceinline__ void patch_moments(long long S1, long long S2, int n, int qc,
                                              float inv_qs, float var_floor, float& dc,
                                              float& sigma) {
  const float inv_n = 1.0f / (float)n;
  const long long ec = S1 - (long long)n * (long long)qc;
  dc = (float)ec * inv_n * inv_qs;
  const long long k = __float2ll_rn((float)S1 * inv_n);
  const unsigned long long uS1 = (unsigned long long)S1, uS2 = (unsigned long long)S2;
  const unsigned long long uk = (unsigned long long)k, un = (unsigned long long)n;
  const unsigned long long T = uS2 - 2ull * uk * uS1 + un * uk * uk;
  const long long e = S1 - (long long)n * k;
  const float ef = (float)e * inv_n;
  const float varq = (float)(long long)T * inv_n - ef * ef;
  const float var = varq * inv_qs * inv_qs;
  sigma = var > var_floor ? sqrtf(var) : 0.0f;
}

template <int MODE, int TX, int TY>
__global__ void __launch_bounds__(kThreads) k_box_pass(BoxArgs a) {
  if (a.stop != nullptr && *(volatile const int*)a.stop != 0) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const BoxLayout L = box_layout(MODE, TX, TY, a.hx, a.hy, a.hz);
  long long* s2z = reinterpret_cast<long long*>(smem + L.o_s2z);
  long long* xb1 = reinterpret_cast<long long*>(smem + L.o_xb1);
  long long* xb2 = reinterpret_cast<long long*>(smem + L.o_xb2);
  int* s1z = reinterpret_cast<int*>(smem + L.o_s1z);
  float* dring = reinterpret_cast<float*>(smem + L.o_dring);

  constexpr int ext = (MODE == kModeIterate) ? 1 : 0;
  const int tid = threadIdx.x;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int hx = a.hx, hy = a.hy, hz = a.hz;
  const size_t plane = (size_t)nx * ny;
  const size_t N = plane * nz;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int z0 = blockIdx.z * a.zlen;
  const int z1 = min(nz, z0 + a.zlen);
  const int WN = L.WN, FN = L.FN, WX = L.WX, FX = L.FX, FY = L.FY;
  const float* __restrict__ src = a.src;

  for (int e = tid; e < WN; e += kThreads) {
    s1z[e] = 0;
    s2z[e] = 0;
  }
  __syncthreads();

  const int zc_lo = max(0, z0 - ext);
  const int zc_hi = min(nz - 1, z1 - 1 + ext);
  const int zi0 = max(0, zc_lo - hz);
  const int zi1 = zc_hi + hz;   // planes past the volume only slide the window out
  float acc0 = 0.0f, acc1 = 0.0f;

  for (int zi = zi0; zi <= zi1; ++zi) {
    // ---- stage 1: z sliding sums of q and q^2 per W column ------------------
    const int zold = zi - L.PZ;            // plane leaving the window
    const bool has_new = zi < nz;
    const bool has_old = zold >= zi0;      // it entered earlier (and is in the volume)
    for (int e = tid; e < WN; e += kThreads) {
      const int wy = e / WX, wx = e - wy * WX;
      const int gx = x0 - ext - hx + wx, gy = y0 - ext - hy + wy;
      if (gx < 0 || gx >= nx || gy < 0 || gy >= ny) continue;   // stays 0
      const size_t g = (size_t)gy * nx + gx;
      int dq1 = 0;
      long long dq2 = 0;
      if (has_new) {
        const int q = __float2int_rn(__ldg(src + (size_t)zi * plane + g) * a.qscale);
        dq1 = q;
        dq2 = (long long)q * q;
      }
      if (has_old) {
        const int q = __float2int_rn(__ldg(src + (size_t)zold * plane + g) * a.qscale);
        dq1 -= q;
        dq2 -= (long long)q * q;
      }
      s1z[e] += dq1;
      s2z[e] += dq2;
    }
    __syncthreads();

    const int zc = zi - hz;
    if (zc < zc_lo || zc > zc_hi) continue;   // uniform across the CTA
    // ---- stage 2a: x window sums by sliding, one task per (row, segment) -----
    for (int t = tid; t < L.WY * L.nsegx; t += kThreads) {
      const int wy = t / L.nsegx, sg = t - wy * L.nsegx;
      const int fx0 = sg * L.segx;
      const int fx1 = min(FX, fx0 + L.segx);
      const int* r1 = s1z + wy * WX;
      const long long* r2 = s2z + wy * WX;
      long long b1 = 0, b2 = 0;
      for (int k = 0; k <= 2 * hx; ++k) {
        b1 += r1[fx0 + k];
        b2 += r2[fx0 + k];
      }
      long long* o1 = xb1 + wy * FX;
      long long* o2 = xb2 + wy * FX;
      o1[fx0] = b1;
      o2[fx0] = b2;
      for (int fx = fx0 + 1; fx < fx1; ++fx) {
        b1 += r1[fx + 2 * hx] - r1[fx - 1];
        b2 += r2[fx + 2 * hx] - r2[fx - 1];
        o1[fx] = b1;
        o2[fx] = b2;
      }
    }
    __syncthreads();
    // ---- stage 2b: y window sums by sliding, moments, correction -------------
    const int nzc = box_count(zc, nz, hz);
    const bool out_plane = (zc >= z0 && zc < z1);
    for (int t = tid; t < FX * L.nsegy; t += kThreads) {
      const int sg = t / FX, fx = t - sg * FX;
      const int fy0 = sg * L.segy;
      const int fy1 = min(FY, fy0 + L.segy);
      const int gx = x0 - ext + fx;
      if (gx < 0 || gx >= nx) continue;
      const int nxc = box_count(gx, nx, hx);
      long long b1 = 0, b2 = 0;
      for (int k = 0; k <= 2 * hy; ++k) {
        b1 += xb1[(fy0 + k) * FX + fx];
        b2 += xb2[(fy0 + k) * FX + fx];
      }
      for (int fy = fy0; fy < fy1; ++fy) {
        if (fy > fy0) {
          b1 += xb1[(fy + 2 * hy) * FX + fx] - xb1[(fy - 1) * FX + fx];
          b2 += xb2[(fy + 2 * hy) * FX + fx] - xb2[(fy - 1) * FX + fx];
        }
        const int gy = y0 - ext + fy;
        if (gy < 0 || gy >= ny) continue;
        const int n = nxc * box_count(gy, ny, hy) * nzc;
        const size_t g = (size_t)zc * plane + (size_t)gy * nx + gx;
        const float vc = __ldg(src + g);
        const int qc = __float2int_rn(vc * a.qscale);
        float dc, sg_;
        patch_moments(b1, b2, n, qc, a.inv_qscale, a.var_floor, dc, sg_);
        if (MODE == kModeStatic) {
          a.out[g] = sg_ > 0.0f ? -dc / sg_ : 0.0f;   // (I_s - E(S)) / STD(S)
          if (a.sd_out) a.sd_out[g] = sg_;
          continue;
        }
        const float zsv = __ldg(a.zs + g);
        const float d = fmaf(zsv, sg_, dc);            // I'_s - I_m^(k)
        if (MODE == kModeIterate) {
          dring[(zc % 3) * FN + fy * FX + fx] = d;
          const bool inner = fx >= 1 && fx <= TX && fy >= 1 && fy <= TY;
          if (inner && out_plane && a.f_tap) a.f_tap[g] = d;
        } else if (MODE == kModeMaskAB) {
          mask_epilogue(a, g, vc, dc, sg_, zsv);
        } else if (MODE == kModeCorrected) {
          a.out[g] = vc + d;
        } else if (MODE == kModeSsdLoss) {
          acc0 = fmaf(d, d, acc0);
        } else if (MODE == kModeSsdAdjoint) {
          // L = sum (m - f)^2: D = dL/dm direct; A, B, C the patch-sum coefficients
          acc0 = fmaf(d, d, acc0);                       // the loss, when partials are given
          const float D = -2.0f * d;
          const float inv_n = 1.0f / (float)n;
          const float A = -D * inv_n;
          const float B = sg_ > 0.0f ? -D * zsv * inv_n / sg_ : 0.0f;
          a.out[g] = A;
          a.out[N + g] = B;
          a.out[2 * N + g] = B * (vc + dc);
          a.out[3 * N + g] = D;
        }
      }
    }
    if (MODE != kModeIterate) continue;
    __syncthreads();
    // ---- stage 3: demons force and update -------------------------------------
    for (int zo = zc - 1; zo <= zc; ++zo) {
      if (zo < z0 || zo >= z1) continue;
      if (zo == zc && zc != nz - 1) continue;
      const float* dp = dring + (zo % 3) * FN;
      const float* dm = dring + ((zo + 2) % 3) * FN;
      const float* dn = dring + ((zo + 1) % 3) * FN;
      for (int e = tid; e < TX * TY; e += kThreads) {
        const int oy = e / TX, ox = e - oy * TX;
        const int gx = x0 + ox, gy = y0 + oy;
        if (gx >= nx || gy >= ny) continue;
        const int fi = (oy + 1) * FX + (ox + 1);
        const size_t g = (size_t)zo * plane + (size_t)gy * nx + gx;
        const float d0 = dp[fi];
        const float m0 = __ldg(src + g);
        // neighbours (clamped reads: one-sided differences at the faces)
        const float mxm = gx > 0 ? __ldg(src + g - 1) : m0;
        const float mxp = gx < nx - 1 ? __ldg(src + g + 1) : m0;
        const float mym = gy > 0 ? __ldg(src + g - nx) : m0;
        const float myp = gy < ny - 1 ? __ldg(src + g + nx) : m0;
        const float mzm = zo > 0 ? __ldg(src + g - plane) : m0;
        const float mzp = zo < nz - 1 ? __ldg(src + g + plane) : m0;
        // neighbours at the faces fall back to the voxel itself (one-sided differences)
        const float dxm = gx > 0 ? dp[fi - 1] : d0, dxp = gx < nx - 1 ? dp[fi + 1] : d0;
        const float dym = gy > 0 ? dp[fi - FX] : d0, dyp = gy < ny - 1 ? dp[fi + FX] : d0;
        const float dzm = zo > 0 ? dm[fi] : d0, dzp = zo < nz - 1 ? dn[fi] : d0;
        const Dr dr = demons_dr(d0, diff_scale(gx, nx), dxp - dxm, mxp - mxm, diff_scale(gy, ny), dyp - dym,
                                myp - mym, diff_scale(zo, nz), dzp - dzm, mzp - mzm,
                                a.force_mode == DISC_FORCE_DOUBLE);
        const float drx = dr.x, dry = dr.y, drz = dr.z;
        const float rx = __ldg(a.r + g), ry = __ldg(a.r + N + g), rz = __ldg(a.r + 2 * N + g);
        const float keep = a.u_is_dr ? 0.0f : 1.0f;   // u = r + dr, or dr alone
        a.out[g] = fmaf(keep, rx, drx);
        a.out[N + g] = fmaf(keep, ry, dry);
        a.out[2 * N + g] = fmaf(keep, rz, drz);
        const bool nin = a.norm_hi <= a.norm_lo || (zo >= a.norm_lo && zo < a.norm_hi);   // the plane enters the norm sums
        acc0 += nin ? norm3(drx, dry, drz) : 0.0f;
        acc1 += nin ? norm3(rx, ry, rz) : 0.0f;
      }
    }
    // the next plane's stage 1 and 2a do not touch the d ring; stage 2b's write
    // of the ring slot read above comes after two more barriers
  }

  if (MODE == kModeIterate || MODE == kModeSsdLoss || MODE == kModeSsdAdjoint) {
    // fixed-order CTA reduction: warp shuffles, then thread 0 over the warp sums
    __shared__ float red[2][kThreads / 32];
    for (int off = 16; off > 0; off >>= 1) {
      acc0 += __shfl_down_sync(0xffffffffu, acc0, off);
      acc1 += __shfl_down_sync(0xffffffffu, acc1, off);
    }
    const int lane = tid & 31, wid = tid >> 5;
    if (lane == 0) {
      red[0][wid] = acc0;
      red[1][wid] = acc1;
    }
    __syncthreads();
    if (tid == 0 && a.partials != nullptr) {
      float s0 = 0.0f, s1 = 0.0f;
      for (int w = 0; w < kThreads / 32; ++w) {
        s0 += red[0][w];
        s1 += red[1][w];
      }
      const size_t b = (size_t)blockIdx.x + (size_t)gridDim.x * (blockIdx.y + (size_t)gridDim.y * blockIdx.z);
      a.partials[2 * b] = s0;
      a.partials[2 * b + 1] = s1;
    }
  }
}

namespace {
constexpr int kTX = 32;
constexpr int kTY = 16;
constexpr size_t kMaxSmem = 226 * 1024;   // leaves room for the static reduction buffer
constexpr size_t kSmemPerSM = 228 * 1024;

// Opt-in dynamic shared memory, raised once per device and kernel instance
// (set_images launches the static mode before any graph capture).
constexpr int kMaxDevices = 64;
int g_smem_set[kMaxDevices][5] = {};

template <int MODE>
cudaError_t launch_mode(const BoxArgs& a, const BoxPlan& p, cudaStream_t s) {
  auto fn = k_box_pass<MODE, kTX, kTY>;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  if ((int)p.smem > g_smem_set[dev][MODE]) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
    if (e != cudaSuccess) return e;
    g_smem_set[dev][MODE] = (int)kMaxSmem;
  }
  fn<<<p.grid, kThreads, p.smem, s>>>(a);
  return cudaGetLastError();
}
}  // namespace

BoxPlan box_plan(int mode, int nx, int ny, int nz, int hx, int hy, int hz, int num_sms) {
  BoxPlan p;
  p.tx = kTX;
  p.ty = kTY;
  p.fast = box_fast_ok(nx, ny, nz, hx, hy, hz);
  p.tma = p.fast && box_tma_ok(mode, nx, ny, nz, hx, hy, hz);
  int per_sm;
  if (p.tma) {
    p.smem = box_tma_smem(mode, hx);
    per_sm = box_tma_occupancy(mode, hx, p.smem);
  } else if (p.fast) {
    p.smem = box_fast_smem(mode, hx);
    per_sm = box_fast_occupancy(mode, hx, p.smem);
  } else {
    const BoxLayout L = box_layout(mode, kTX, kTY, hx, hy, hz);
    p.smem = L.total;
    if (p.smem > kMaxSmem) {
      p.grid = dim3(0, 0, 0);
      p.zlen = 0;
      return p;
    }
    per_sm = (int)(kSmemPerSM / (p.smem + 1024));
  }
  const int gx = (nx + kTX - 1) / kTX, gy = (ny + kTY - 1) / kTY;
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 8) per_sm = 8;                 // 8 CTAs of 256 threads fill an SM
  // at most one wave of resident CTAs: fewer, longer z chunks amortise the z
  // halo, and a partial second wave would double the time of the first
  const long long slots = (long long)num_sms * per_sm;
  long long chunks = slots / ((long long)gx * gy);
  if (chunks < 1) chunks = 1;
  long long max_chunks = (nz + 1) / 2;       // at least 2 output planes per chunk
  if (max_chunks < 1) max_chunks = 1;
  if (chunks > max_chunks) chunks = max_chunks;
  p.zlen = (int)((nz + chunks - 1) / chunks);
  const int gz = (nz + p.zlen - 1) / p.zlen;
  p.grid = dim3(gx, gy, gz);
  return p;
}

namespace {
// The wide-tile plan where its one wave gets enough planes per CTA to amortise
// the z warm-up of a march (grid.x = 0: not eligible).
BoxPlan wide_plan(int nx, int ny, int nz, int hx, int hy, int hz, int num_sms, bool aligned,
                  int min_planes = kWideMinPlanes) {
  BoxPlan none{};
  none.grid = dim3(0, 0, 0);
  if (aligned && box_wide_ok(nx, ny, nz, hx, hy, hz)) {
    int tx = 0, ty = 0;
    box_wide_tile(&tx, &ty);
    const int occ = box_wide_occupancy(hx);
    const long long slots = (long long)num_sms * (occ < 1 ? 1 : occ);
    const long long P = (long long)((nx + tx - 1) / tx) * ((ny + ty - 1) / ty) * nz;
    if (occ >= 1 && (P >= (long long)min_planes * slots || (test_switches() & DISC_SW_WIDE_ANY))) {
      BoxPlan p;
      p.tx = tx;
      p.ty = ty;
      p.fast = p.tma = p.wide = true;
      p.smem = box_wide_smem(hx);
      p.zlen = nz;
      p.grid = dim3((unsigned)slots, 1, 1);
      return p;
    }
  }
  return none;
}
}  // namespace

BoxPlan box_plan_iter(int nx, int ny, int nz, int hx, int hy, int hz, int num_sms, const float* src,
                      const float* r, const float* u) {
  const bool aligned = (((uintptr_t)src | (uintptr_t)r | (uintptr_t)u) & 15u) == 0u;
  const BoxPlan w = wide_plan(nx, ny, nz, hx, hy, hz, num_sms, aligned);
  return w.grid.x != 0 ? w : box_plan(kModeIterate, nx, ny, nz, hx, hy, hz, num_sms);
}

BoxPlan box_plan_wide_mode(int mode, int nx, int ny, int nz, int hx, int hy, int hz, int num_sms,
                           const float* src, const float* out) {
  const bool aligned = (((uintptr_t)src | (uintptr_t)out) & 15u) == 0u;
  const BoxPlan w = wide_plan(nx, ny, nz, hx, hy, hz, num_sms, aligned,
                              mode == kModeMaskAB ? kWideMinPlanesMask : kWideMinPlanes);
  return w.grid.x != 0 ? w : box_plan(mode, nx, ny, nz, hx, hy, hz, num_sms);
}

cudaError_t box_launch(int mode, const BoxArgs& a, const BoxPlan& p, cudaStream_t s) {
  if (p.grid.x == 0) return cudaErrorInvalidConfiguration;
  if (p.wide) return box_wide_launch(mode, a, p, s);
  BoxArgs b = a;
  b.zlen = p.zlen;
  if (p.tma) {
    if (box_tma_aligned(mode, b)) return box_tma_launch(mode, b, p, s);
    BoxPlan q = p;                            // unaligned buffers: same grid, plain loads
    q.smem = box_fast_smem(mode, a.hx);
    return box_fast_launch(mode, b, q, s);
  }
  if (p.fast) return box_fast_launch(mode, b, p, s);
  switch (mode) {
    case kModeStatic: return launch_mode<kModeStatic>(b, p, s);
    case kModeIterate: return launch_mode<kModeIterate>(b, p, s);
    case kModeCorrected: return launch_mode<kModeCorrected>(b, p, s);
    case kModeSsdLoss: return launch_mode<kModeSsdLoss>(b, p, s);
    case kModeSsdAdjoint: return launch_mode<kModeSsdAdjoint>(b, p, s);
    case kModeMaskAB: return launch_mode<kModeMaskAB>(b, p, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace disc
