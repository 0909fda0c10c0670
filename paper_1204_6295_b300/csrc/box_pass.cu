// Warp + patch-moment kernels of the DISC iteration (sm_103a).
//
// One z-marching CTA owns a TX x TY column tile of output voxels and a chunk of
// z planes.  For every plane it enters it
//   1. evaluates the plane's values on the tile plus the patch halo: the
//      moving image warped by the field, m = I_m(x + r(x)) (Sec. 2.1; Sec. 2.3
//      kernel 5), or the CBCT itself for the static statistics;
//   2. quantises them to q = rint(v * 2^e) and keeps exact integer patch sums
//      sum q and sum q^2: a sliding window over z (ring of the last P_z planes
//      in shared memory), then direct sums over x and y;
//   3. turns the sums into the patch moments E(X), STD(X) of Eq. (3) and the
//      Appendix (A.4), and from them the moment-matched CBCT
//      f = I'_s = zs STD(M) + E(M), which equals a I_s + b of Eqs. (5)-(6)
//      with zs = (I_s - E(S)) / STD(S);
//   4. (iteration mode) from a ring of three f planes and the kept m planes,
//      the gradient of I'_s (central differences, one-sided at the faces), the
//      demons force of Eq. (1) and u = r + dr (Algorithm A1 steps 4 and 5),
//      with per-CTA sums of |dr| and |r| for the Sec. 2.3 stopping norm.
//
// Integer sums make the statistics exact and independent of tile shape and
// order: a constant patch has variance exactly 0 and the plain and batched
// launches give bit-identical results.

#include <cuda_runtime.h>

#include "internal.cuh"

namespace disc {

struct BoxLayout {
  int WX, WY, FX, FY, PZ, MR, WN, FN;
  size_t o_s2z, o_xb1, o_xb2, o_qring, o_s1z, o_fring, o_mring, total;
};

// Shared-memory layout of a box-pass CTA.  The F region is the tile plus a
// one-voxel ring in iteration mode (the gradient of I'_s needs it); the W region
// adds the patch half sizes around F.
__host__ __device__ inline BoxLayout box_layout(int mode, int TX, int TY, int hx, int hy, int hz) {
  BoxLayout L;
  const int ext = (mode == kModeIterate) ? 1 : 0;
  L.FX = TX + 2 * ext;
  L.FY = TY + 2 * ext;
  L.WX = L.FX + 2 * hx;
  L.WY = L.FY + 2 * hy;
  L.PZ = 2 * hz + 1;
  L.MR = (mode == kModeIterate) ? hz + 3 : hz + 1;
  L.WN = L.WX * L.WY;
  L.FN = L.FX * L.FY;
  size_t o = 0;
  L.o_s2z = o;   o += 8 * (size_t)L.WN;
  L.o_xb1 = o;   o += 8 * (size_t)(L.FX * L.WY);
  L.o_xb2 = o;   o += 8 * (size_t)(L.FX * L.WY);
  L.o_qring = o; o += 4 * (size_t)L.PZ * L.WN;
  L.o_s1z = o;   o += 4 * (size_t)L.WN;
  L.o_fring = o; o += (mode == kModeIterate) ? 4 * 3 * (size_t)L.FN : 0;
  L.o_mring = o; o += 4 * (size_t)L.MR * L.FN;
  L.total = (o + 15) & ~(size_t)15;
  return L;
}

// Trilinear sample position along one axis: voxel c displaced by rv, clamped to
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

// m = I_m(x + r(x)) by trilinear interpolation (Sec. 2.1, Sec. 2.3 kernel 5).
__device__ __forceinline__ float warp_at(const float* __restrict__ Im, int x, int y, int z,
                                         float rx, float ry, float rz, int nx, int ny, int nz) {
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

// Patch moments from exact integer sums of q = rint(v 2^e) over n voxels.
//  mu    = v_c + (S1 - n q_c) / (n 2^e): the quantised mean, re-anchored on the
//          exact centre value so that a constant patch returns its value exactly.
//  sigma = sqrt(Var) with Var = (T/n - (e/n)^2) / 2^(2e),
//          T = sum (q - k)^2 = S2 - 2 k S1 + n k^2, k = round(S1/n), e = S1 - n k,
//          evaluated modulo 2^64 (the true T fits in 63 bits), so no precision is
//          lost to the cancellation of E(X^2) - E(X)^2.  sigma = 0 when
//          Var <= var_floor.
//  dev_c = v_c - mu.
__device__ __forceinline__ void patch_moments(long long S1, long long S2, int n, int qc, float vc,
                                              float inv_qs, float var_floor, float& mu,
                                              float& sigma, float& dev_c) {
  const float inv_n = 1.0f / (float)n;
  const long long ec = S1 - (long long)n * (long long)qc;
  const float dc = (float)ec * inv_n * inv_qs;
  mu = vc + dc;
  dev_c = -dc;
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

// Gradient of a plane-ring quantity at F index fi along x and y (in-plane).
__device__ __forceinline__ float grad_axis(const float* p, int fi, int stride, int c, int n) {
  if (n < 2) return 0.0f;
  if (c == 0) return p[fi + stride] - p[fi];
  if (c == n - 1) return p[fi] - p[fi - stride];
  return 0.5f * (p[fi + stride] - p[fi - stride]);
}
__device__ __forceinline__ float grad_z(const float* ring, int FN, int nring, int fi, int z, int nz) {
  if (nz < 2) return 0.0f;
  const float* pm = ring + ((z + nring - 1) % nring) * FN;
  const float* p0 = ring + (z % nring) * FN;
  const float* pp = ring + ((z + 1) % nring) * FN;
  if (z == 0) return pp[fi] - p0[fi];
  if (z == nz - 1) return p0[fi] - pm[fi];
  return 0.5f * (pp[fi] - pm[fi]);
}

template <int MODE, int TX, int TY>
__global__ void __launch_bounds__(kThreads) k_box_pass(BoxArgs a) {
  if (a.stop != nullptr && *(volatile const int*)a.stop != 0) return;
  extern __shared__ __align__(16) unsigned char smem[];
  const BoxLayout L = box_layout(MODE, TX, TY, a.hx, a.hy, a.hz);
  long long* s2z = reinterpret_cast<long long*>(smem + L.o_s2z);
  long long* xb1 = reinterpret_cast<long long*>(smem + L.o_xb1);
  long long* xb2 = reinterpret_cast<long long*>(smem + L.o_xb2);
  int* qring = reinterpret_cast<int*>(smem + L.o_qring);
  int* s1z = reinterpret_cast<int*>(smem + L.o_s1z);
  float* fring = reinterpret_cast<float*>(smem + L.o_fring);
  float* mring = reinterpret_cast<float*>(smem + L.o_mring);

  constexpr int ext = (MODE == kModeIterate) ? 1 : 0;
  const int tid = threadIdx.x;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int hx = a.hx, hy = a.hy, hz = a.hz;
  const size_t N = (size_t)nx * ny * nz;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const int z0 = blockIdx.z * a.zlen;
  const int z1 = min(nz, z0 + a.zlen);
  const int WN = L.WN, FN = L.FN, WX = L.WX, FX = L.FX;

  for (int e = tid; e < L.PZ * WN; e += kThreads) qring[e] = 0;
  for (int e = tid; e < WN; e += kThreads) {
    s1z[e] = 0;
    s2z[e] = 0;
  }
  __syncthreads();

  const int zc_lo = max(0, z0 - ext);
  const int zc_hi = min(nz - 1, z1 - 1 + ext);
  const int zi0 = max(0, zc_lo - hz);
  const int zi1 = zc_hi + hz;   // planes >= nz enter as zeros to slide the window out
  float acc0 = 0.0f, acc1 = 0.0f;

  for (int zi = zi0; zi <= zi1; ++zi) {
    const int slot = (zi - zi0) % L.PZ;
    const bool plane_in = zi < nz;
    // ---- stage 1: plane values on the W region, z sliding sums --------------
    for (int e = tid; e < WN; e += kThreads) {
      const int wy = e / WX, wx = e - wy * WX;
      const int gx = x0 - ext - hx + wx, gy = y0 - ext - hy + wy;
      float v = 0.0f;
      int q = 0;
      if (plane_in && gx >= 0 && gx < nx && gy >= 0 && gy < ny) {
        const size_t g = vix(gx, gy, zi, nx, ny);
        if (MODE == kModeStatic) {
          v = __ldg(a.src + g);
        } else {
          v = warp_at(a.src, gx, gy, zi, __ldg(a.r + g), __ldg(a.r + N + g), __ldg(a.r + 2 * N + g),
                      nx, ny, nz);
        }
        q = __float2int_rn(v * a.qscale);
      }
      int* qs = qring + slot * WN + e;
      const int qo = *qs;
      *qs = q;
      s1z[e] += q - qo;
      s2z[e] += (long long)q * q - (long long)qo * qo;
      const int fx = wx - hx, fy = wy - hy;
      if (fx >= 0 && fx < FX && fy >= 0 && fy < L.FY && zi < nz)
        mring[(zi % L.MR) * FN + fy * FX + fx] = v;
    }
    __syncthreads();

    const int zc = zi - hz;
    if (zc >= zc_lo && zc <= zc_hi) {
      // ---- stage 2a: x box sums over the F columns ---------------------------
      const int XN = FX * L.WY;
      for (int e = tid; e < XN; e += kThreads) {
        const int wy = e / FX, fx = e - wy * FX;
        const int* r1 = s1z + wy * WX + fx;
        const long long* r2 = s2z + wy * WX + fx;
        long long b1 = 0, b2 = 0;
        for (int k = 0; k <= 2 * hx; ++k) {
          b1 += r1[k];
          b2 += r2[k];
        }
        xb1[e] = b1;
        xb2[e] = b2;
      }
      __syncthreads();
      // ---- stage 2b: y box sums, moments, correction ---------------------------
      const int cslot = (zc - zi0) % L.PZ;
      const int nzc = box_count(zc, nz, hz);
      const bool out_plane = (zc >= z0 && zc < z1);
      for (int e = tid; e < FN; e += kThreads) {
        const int fy = e / FX, fx = e - fy * FX;
        const int gx = x0 - ext + fx, gy = y0 - ext + fy;
        if (gx < 0 || gx >= nx || gy < 0 || gy >= ny) continue;
        long long S1 = 0, S2 = 0;
        for (int k = 0; k <= 2 * hy; ++k) {
          S1 += xb1[(fy + k) * FX + fx];
          S2 += xb2[(fy + k) * FX + fx];
        }
        const int n = box_count(gx, nx, hx) * box_count(gy, ny, hy) * nzc;
        const int qc = qring[cslot * WN + (fy + hy) * WX + (fx + hx)];
        const float vc = mring[(zc % L.MR) * FN + e];
        float mu, sg, dev;
        patch_moments(S1, S2, n, qc, vc, a.inv_qscale, a.var_floor, mu, sg, dev);
        const size_t g = vix(gx, gy, zc, nx, ny);
        if (MODE == kModeStatic) {
          a.out[g] = sg > 0.0f ? dev / sg : 0.0f;
          continue;
        }
        const float zsv = __ldg(a.zs + g);
        const float f = fmaf(zsv, sg, mu);
        if (MODE == kModeIterate) {
          fring[(zc % 3) * FN + e] = f;
          const bool inner = fx >= 1 && fx <= TX && fy >= 1 && fy <= TY;
          if (inner && out_plane) {
            if (a.f_tap) a.f_tap[g] = f;
            if (a.m_tap) a.m_tap[g] = vc;
          }
        } else if (MODE == kModeCorrected) {
          a.out[g] = f;
        } else if (MODE == kModeSsdLoss) {
          const float d = vc - f;
          acc0 = fmaf(d, d, acc0);
        } else if (MODE == kModeSsdAdjoint) {
          // L = sum (m - f)^2; D = dL/dm direct, A/B/C the patch-sum coefficients
          const float D = 2.0f * (vc - f);
          const float inv_n = 1.0f / (float)n;
          const float A = -D * inv_n;
          const float B = sg > 0.0f ? -D * zsv * inv_n / sg : 0.0f;
          a.out[g] = A;
          a.out[N + g] = B;
          a.out[2 * N + g] = B * mu;
          a.out[3 * N + g] = D;
        }
      }
      __syncthreads();
      // ---- stage 3: demons force and update (iteration mode) ------------------
      if (MODE == kModeIterate) {
        for (int zo = zc - 1; zo <= zc; ++zo) {
          if (zo < z0 || zo >= z1) continue;
          if (zo == zc && zc != nz - 1) continue;
          for (int e = tid; e < TX * TY; e += kThreads) {
            const int oy = e / TX, ox = e - oy * TX;
            const int gx = x0 + ox, gy = y0 + oy;
            if (gx >= nx || gy >= ny) continue;
            const int fi = (oy + 1) * FX + (ox + 1);
            const float* fp = fring + (zo % 3) * FN;
            const float f = fp[fi];
            const float m = mring[(zo % L.MR) * FN + fi];
            const float gfx = grad_axis(fp, fi, 1, gx, nx);
            const float gfy = grad_axis(fp, fi, FX, gy, ny);
            const float gfz = grad_z(fring, FN, 3, fi, zo, nz);
            const float diff = f - m;
            const float d2 = diff * diff;
            const float den = fmaf(gfx, gfx, fmaf(gfy, gfy, fmaf(gfz, gfz, d2)));
            const float s = den > 1e-9f ? diff / den : 0.0f;
            float drx = s * gfx, dry = s * gfy, drz = s * gfz;
            if (a.force_mode == DISC_FORCE_DOUBLE) {
              const float* mp = mring + (zo % L.MR) * FN;
              const float gmx = grad_axis(mp, fi, 1, gx, nx);
              const float gmy = grad_axis(mp, fi, FX, gy, ny);
              const float gmz = grad_z(mring, FN, L.MR, fi, zo, nz);
              const float den2 = fmaf(gmx, gmx, fmaf(gmy, gmy, fmaf(gmz, gmz, d2)));
              const float s2 = den2 > 1e-9f ? diff / den2 : 0.0f;
              drx = fmaf(s2, gmx, drx);
              dry = fmaf(s2, gmy, dry);
              drz = fmaf(s2, gmz, drz);
            }
            const size_t g = vix(gx, gy, zo, nx, ny);
            const float rx = __ldg(a.r + g), ry = __ldg(a.r + N + g), rz = __ldg(a.r + 2 * N + g);
            a.out[g] = rx + drx;
            a.out[N + g] = ry + dry;
            a.out[2 * N + g] = rz + drz;
            acc0 += sqrtf(fmaf(drx, drx, fmaf(dry, dry, drz * drz)));
            acc1 += sqrtf(fmaf(rx, rx, fmaf(ry, ry, rz * rz)));
          }
        }
      }
    }
    __syncthreads();
  }

  if (MODE == kModeIterate || MODE == kModeSsdLoss) {
    // fixed-order CTA reduction: warp shuffles, then warp 0 over the warp sums
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
    if (tid == 0) {
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

// Opt-in dynamic shared memory, raised once per device and kernel instance
// (outside any stream capture, since set_images launches every mode first).
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
  const BoxLayout L = box_layout(mode, kTX, kTY, hx, hy, hz);
  p.smem = L.total;
  if (p.smem > kMaxSmem) {
    p.grid = dim3(0, 0, 0);
    p.zlen = 0;
    return p;
  }
  const int gx = (nx + kTX - 1) / kTX, gy = (ny + kTY - 1) / kTY;
  int per_sm = (int)(kMaxSmem / (p.smem + 1024));
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 8) per_sm = 8;
  const long long target = 2LL * num_sms * per_sm;   // about two waves of resident CTAs
  long long chunks = (target + (long long)gx * gy - 1) / ((long long)gx * gy);
  if (chunks < 1) chunks = 1;
  // keep at least 4 output planes per chunk unless the volume is thinner
  long long max_chunks = (nz + 3) / 4;
  if (max_chunks < 1) max_chunks = 1;
  if (chunks > max_chunks) chunks = max_chunks;
  p.zlen = (int)((nz + chunks - 1) / chunks);
  const int gz = (nz + p.zlen - 1) / p.zlen;
  p.grid = dim3(gx, gy, gz);
  return p;
}

cudaError_t box_launch(int mode, const BoxArgs& a, const BoxPlan& p, cudaStream_t s) {
  if (p.grid.x == 0) return cudaErrorInvalidConfiguration;
  BoxArgs b = a;
  b.zlen = p.zlen;
  switch (mode) {
    case kModeStatic: return launch_mode<kModeStatic>(b, p, s);
    case kModeIterate: return launch_mode<kModeIterate>(b, p, s);
    case kModeCorrected: return launch_mode<kModeCorrected>(b, p, s);
    case kModeSsdLoss: return launch_mode<kModeSsdLoss>(b, p, s);
    case kModeSsdAdjoint: return launch_mode<kModeSsdAdjoint>(b, p, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace disc
