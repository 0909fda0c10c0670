// Patch-moment kernels specialised for cubic patches of half size H (patch
// 2H+1 per axis, H = 1..7) on a 32 x 16 column tile (sm_103a).
//
// Same computation as the generic box pass (box_pass.cu): exact integer
// sliding sums of q = rint(v 2^e) and q^2 over the truncated patch (Eq. 3),
// the patch moments E(X), STD(X) (Appendix A.4), the moment-matched CBCT kept
// as d = I'_s - I_m^(k) = zs STD(M) + (E(M) - m) (Eqs. 5-6), and in iteration
// mode the demons force of Eq. (1) with grad I'_s = grad d + grad m and the
// update u = r + dr (Algorithm A1 steps 3-5).  With every size known at
// compile time the index arithmetic uses constant divisors, the per-column z
// sums live in registers, the leaving plane is re-read from L2 instead of
// being kept in shared memory, and the x and y window sums slide.

#include <cuda_runtime.h>

#include "box_dev.cuh"
#include "internal.cuh"

namespace disc {

namespace {

template <int MODE, int H>
struct FastLayout {
  static constexpr int EXT = (MODE == kModeIterate) ? 1 : 0;
  static constexpr int TX = 32, TY = 16;
  static constexpr int FX = TX + 2 * EXT, FY = TY + 2 * EXT;
  static constexpr int WX = FX + 2 * H, WY = FY + 2 * H;
  static constexpr int WXP = WX | 1;                     // odd row stride of the z-sum plane
  static constexpr int WN = WX * WY;
  static constexpr int K1 = (WN + kThreads - 1) / kThreads;   // W columns per thread
  static constexpr int FN = FX * FY;
  // sliding tasks: about one per thread (short tasks keep every warp busy)
  static constexpr int NSX0 = (kThreads / WY) < 1 ? 1 : (kThreads / WY);
  static constexpr int SX = (FX + NSX0 - 1) / NSX0;     // x outputs per sliding task
  static constexpr int NSX = (FX + SX - 1) / SX;
  static constexpr int NSY0 = (kThreads / FX) < 1 ? 1 : (kThreads / FX);
  static constexpr int SY = (FY + NSY0 - 1) / NSY0;     // y outputs per sliding task
  static constexpr int NSY = (FY + SY - 1) / SY;
  static constexpr int KF = (FN + kThreads - 1) / kThreads;      // F elements per thread
  static constexpr int TN = TX * TY;
  static constexpr int KO = (TN + kThreads - 1) / kThreads;      // tile elements per thread
  static constexpr int NP = (2 * H + 1) * (2 * H + 1) * (2 * H + 1);
  static constexpr size_t o_s2z = 0;
  static constexpr size_t o_xb1 = o_s2z + 8 * (size_t)WY * WXP;
  static constexpr size_t o_xb2 = o_xb1 + 8 * (size_t)WY * FX;
  static constexpr size_t o_s1z = o_xb2 + 8 * (size_t)WY * FX;
  static constexpr size_t o_dring = o_s1z + 4 * (size_t)WY * WXP;
  static constexpr size_t o_mring = o_dring + (EXT ? 4 * 3 * (size_t)FN : 0);
  static constexpr size_t o_zsf = o_mring + 4 * (EXT ? 3 : 1) * (size_t)FN;   // zs of the centre plane
  static constexpr size_t o_ro = o_zsf + (MODE == kModeStatic ? 0 : 4 * (size_t)FN);
  static constexpr size_t bytes = ((o_ro + (EXT ? 4 * 3 * (size_t)TN : 0)) + 15) & ~(size_t)15;
};



// The CTA body: tile (bx, by) of the 32 x 16 tiling, z chunk bz; part = index
// of this CTA's norm partials.  Shared by the per-volume and batched launches.
template <int MODE, int H>
__device__ __forceinline__ void box_body(const BoxArgs& a, int bx, int by, int bz, size_t part) {
  using B = FastLayout<MODE, H>;
  if (a.stop != nullptr && *(volatile const int*)a.stop != 0) return;
  extern __shared__ __align__(16) unsigned char smem[];
  long long* s2z = reinterpret_cast<long long*>(smem + B::o_s2z);
  long long* xb1 = reinterpret_cast<long long*>(smem + B::o_xb1);
  long long* xb2 = reinterpret_cast<long long*>(smem + B::o_xb2);
  int* s1z = reinterpret_cast<int*>(smem + B::o_s1z);
  float* dring = reinterpret_cast<float*>(smem + B::o_dring);
  float* mring = reinterpret_cast<float*>(smem + B::o_mring);   // v on the F region (3 planes if EXT)
  float* zsf = reinterpret_cast<float*>(smem + B::o_zsf);       // zs on the F region, centre plane
  float* ro = reinterpret_cast<float*>(smem + B::o_ro);         // r on the tile, force plane
  constexpr int NMR = B::EXT ? 3 : 1;

  const int tid = threadIdx.x;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int plane = nx * ny;                 // 3 N < 2^31 is checked on the host
  const int N = plane * nz;
  const int x0 = bx * B::TX, y0 = by * B::TY;
  const int z0 = bz * a.zlen;
  const int z1 = min(nz, z0 + a.zlen);
  const float* __restrict__ src = a.src;
  const float qs = a.qscale, inv_qs = a.inv_qscale, vfl = a.var_floor;

  // ---- per-thread element maps (fixed for the whole march) -------------------
  // W columns: plane offset (or -1 outside) and smem index; running z sums
  int goff[B::K1], sidx[B::K1], s1r[B::K1];
  long long s2r[B::K1];
#pragma unroll
  for (int k = 0; k < B::K1; ++k) {
    const int e = tid + k * kThreads;
    goff[k] = -1;
    sidx[k] = -1;
    s1r[k] = 0;
    s2r[k] = 0;
    if (e < B::WN) {
      const int wy = e / B::WX, wx = e - wy * B::WX;
      const int gx = x0 - B::EXT - H + wx, gy = y0 - B::EXT - H + wy;
      sidx[k] = wy * B::WXP + wx;
      if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) goff[k] = gy * nx + gx;
    }
  }
  // F elements: plane offset (or -1)
  int foff[B::KF];
#pragma unroll
  for (int k = 0; k < B::KF; ++k) {
    const int e = tid + k * kThreads;
    foff[k] = -1;
    if (e < B::FN) {
      const int fy = e / B::FX, fx = e - fy * B::FX;
      const int gx = x0 - B::EXT + fx, gy = y0 - B::EXT + fy;
      if (gx >= 0 && gx < nx && gy >= 0 && gy < ny) foff[k] = gy * nx + gx;
    }
  }
  // tile elements: plane offset (or -1)
  int ooff[B::KO];
#pragma unroll
  for (int k = 0; k < B::KO; ++k) {
    const int e = tid + k * kThreads;
    const int oy = e / B::TX, ox = e - oy * B::TX;
    ooff[k] = (e < B::TN && x0 + ox < nx && y0 + oy < ny) ? (y0 + oy) * nx + x0 + ox : -1;
  }

  const int zc_lo = max(0, z0 - B::EXT);
  const int zc_hi = min(nz - 1, z1 - 1 + B::EXT);
  const int zi0 = max(0, zc_lo - H);
  const int zi1 = zc_hi + H;
  float acc0 = 0.0f, acc1 = 0.0f;

  for (int zi = zi0; zi <= zi1; ++zi) {
    const int zc = zi - H;                   // centre plane of the patch window
    const bool do2 = zc >= zc_lo && zc <= zc_hi;
    const int zf = zc - 1;                   // plane whose force is computed this step
    const bool do3 = (MODE == kModeIterate) && do2 && zf >= z0 && zf < z1;
    // ---- stage 1: every global load of this step, issued together ------------
    const int zold = zi - (2 * H + 1);
    const bool has_new = zi < nz, has_old = zold >= zi0;
    const float* pn = src + (size_t)zi * plane;
    const float* po = src + (size_t)(has_old ? zold : 0) * plane;
    float vn[B::K1], vo[B::K1];
#pragma unroll
    for (int k = 0; k < B::K1; ++k) {
      vn[k] = (has_new && goff[k] >= 0) ? ldg_in(src, (long long)(pn - src) + goff[k], N) : 0.0f;
      vo[k] = (has_old && goff[k] >= 0) ? ldg_in(src, (long long)(po - src) + goff[k], N) : 0.0f;
    }
    float fm[B::KF], fz[B::KF];
    if (do2) {
      const float* pc = src + (size_t)zc * plane;
      const float* pz = a.zs + (size_t)zc * plane;
#pragma unroll
      for (int k = 0; k < B::KF; ++k) {
        fm[k] = foff[k] >= 0 ? ldg_in(src, (long long)(pc - src) + foff[k], N) : 0.0f;
        fz[k] = (MODE != kModeStatic && foff[k] >= 0) ? ldg_in(a.zs, (long long)(pz - a.zs) + foff[k], N) : 0.0f;
      }
    }
    float rv[3][B::KO];
    if (do3) {
      const float* pr = a.r + (size_t)zf * plane;
#pragma unroll
      for (int k = 0; k < B::KO; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          rv[c][k] = ooff[k] >= 0 ? ldg_in(a.r, (long long)(pr - a.r) + (long long)c * N + ooff[k], 3LL * N) : 0.0f;
    }
    // z sliding sums
#pragma unroll
    for (int k = 0; k < B::K1; ++k) {
      if (sidx[k] < 0) continue;
      const int qn = __float2int_rn(vn[k] * qs), qo = __float2int_rn(vo[k] * qs);
      s1r[k] += qn - qo;
      s2r[k] += (long long)qn * qn - (long long)qo * qo;
      s1z[sidx[k]] = s1r[k];
      s2z[sidx[k]] = s2r[k];
    }
    if (do2) {
      float* mr = mring + (zc % NMR) * B::FN;
#pragma unroll
      for (int k = 0; k < B::KF; ++k) {
        const int e = tid + k * kThreads;
        if (e < B::FN) {
          mr[e] = fm[k];
          if (MODE != kModeStatic) zsf[e] = fz[k];
        }
      }
    }
    if (do3) {
#pragma unroll
      for (int k = 0; k < B::KO; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) ro[c * B::TN + tid + k * kThreads] = rv[c][k];
    }
    __syncthreads();
    if (!do2) continue;                      // uniform

    // ---- stage 2a: x window sums, sliding, one task per (segment, row) ---------
    for (int t = tid; t < B::NSX * B::WY; t += kThreads) {
      const int sg = t / B::WY, wy = t - sg * B::WY;
      const int fx0 = sg * B::SX;
      const int* r1 = s1z + wy * B::WXP + fx0;
      const long long* r2 = s2z + wy * B::WXP + fx0;
      long long b1 = tree_sum<2 * H + 1, int>(r1, 1), b2 = tree_sum<2 * H + 1, long long>(r2, 1);
      long long* o1 = xb1 + wy * B::FX + fx0;
      long long* o2 = xb2 + wy * B::FX + fx0;
      o1[0] = b1;
      o2[0] = b2;
#pragma unroll
      for (int j = 1; j < B::SX; ++j) {
        if (fx0 + j < B::FX) {
          b1 += r1[j + 2 * H] - r1[j - 1];
          b2 += r2[j + 2 * H] - r2[j - 1];
          o1[j] = b1;
          o2[j] = b2;
        }
      }
    }
    __syncthreads();

    // ---- stage 2b: y window sums, sliding; moments and correction --------------
    const bool zin = zc >= H && zc < nz - H;
    const int nzc = box_count(zc, nz, H);
    const bool out_plane = zc >= z0 && zc < z1;
    const float* mr = mring + (zc % NMR) * B::FN;
    for (int t = tid; t < B::NSY * B::FX; t += kThreads) {
      const int sy = t / B::FX, fx = t - sy * B::FX;
      const int gx = x0 - B::EXT + fx;
      if (gx < 0 || gx >= nx) continue;
      const int fy0 = sy * B::SY;
      const bool xin = gx >= H && gx < nx - H;
      const int nxc = box_count(gx, nx, H);
      long long b1 = tree_sum<2 * H + 1, long long>(xb1 + fy0 * B::FX + fx, B::FX);
      long long b2 = tree_sum<2 * H + 1, long long>(xb2 + fy0 * B::FX + fx, B::FX);
#pragma unroll
      for (int j = 0; j < B::SY; ++j) {
        const int fy = fy0 + j;
        if (fy >= B::FY) break;
        if (j > 0) {
          b1 += xb1[(fy + 2 * H) * B::FX + fx] - xb1[(fy - 1) * B::FX + fx];
          b2 += xb2[(fy + 2 * H) * B::FX + fx] - xb2[(fy - 1) * B::FX + fx];
        }
        const int gy = y0 - B::EXT + fy;
        if (gy < 0 || gy >= ny) continue;
        int n;
        float inv_n;
        if (xin && zin && gy >= H && gy < ny - H) {
          n = B::NP;
          inv_n = 1.0f / (float)B::NP;
        } else {
          n = nxc * box_count(gy, ny, H) * nzc;
          inv_n = 1.0f / (float)n;
        }
        const int fi = fy * B::FX + fx;
        const float vc = mr[fi];
        float dc, sg_;
        patch_moments(b1, b2, n, inv_n, __float2int_rn(vc * qs), inv_qs, vfl, dc, sg_);
        const size_t gz = (size_t)zc * plane + (size_t)gy * nx + gx;
        if (MODE == kModeStatic) {
          st_in(a.out, gz, N, sg_ > 0.0f ? -dc / sg_ : 0.0f);   // (I_s - E(S)) / STD(S)
          if (a.sd_out) a.sd_out[gz] = sg_;
          continue;
        }
        const float zsv = zsf[fi];
        const float d = fmaf(zsv, sg_, dc);               // I'_s - I_m^(k)
        if (MODE == kModeIterate) {
          dring[(zc % 3) * B::FN + fi] = d;
          if (a.f_tap && out_plane && fx >= 1 && fx <= B::TX && fy >= 1 && fy <= B::TY) st_in(a.f_tap, gz, N, d);
        } else if (MODE == kModeMaskAB) {
          mask_epilogue(a, gz, vc, dc, sg_, zsv);
        } else if (MODE == kModeCorrected) {
          st_in(a.out, gz, N, vc + d);
        } else if (MODE == kModeSsdLoss) {
          acc0 = fmaf(d, d, acc0);
        } else if (MODE == kModeSsdAdjoint) {
          acc0 = fmaf(d, d, acc0);                       // the loss, when partials are given
          const float D = -2.0f * d;
          const float A = -D * inv_n;
          const float Bc = sg_ > 0.0f ? -D * zsv * inv_n / sg_ : 0.0f;
          st_in(a.out, gz, 4LL * N, A);
          st_in(a.out, (long long)N + gz, 4LL * N, Bc);
          st_in(a.out, 2LL * N + gz, 4LL * N, Bc * (vc + dc));
          st_in(a.out, 3LL * N + gz, 4LL * N, D);
        }
      }
    }
    if (MODE == kModeIterate) {
    __syncthreads();

    // ---- stage 3: demons force (Eq. 1) and update ------------------------------
#pragma unroll
    for (int back = 1; back >= 0; --back) {
      const int zo = zc - back;
      if (zo < z0 || zo >= z1) continue;
      if (back == 0 && zc != nz - 1) continue;
      const int so = zo % 3, sm = (zo + 2) % 3, sp = (zo + 1) % 3;
      const float* dp = dring + so * B::FN;
      const float* mp = mring + so * B::FN;
      const bool zlo = zo > 0, zhi = zo < nz - 1;
#pragma unroll
      for (int i = 0; i < B::KO; ++i) {
        const int o = tid + i * kThreads;
        if (ooff[i] < 0) continue;
        const int oy = o / B::TX, ox = o - oy * B::TX;
        const int gx = x0 + ox, gy = y0 + oy;
        const int fi = (oy + 1) * B::FX + (ox + 1);
        const float d0 = dp[fi], m0 = mp[fi];
        const int xl = gx > 0 ? -1 : 0, xh = gx < nx - 1 ? 1 : 0;
        const int yl = gy > 0 ? -B::FX : 0, yh = gy < ny - 1 ? B::FX : 0;
        const float dzm = zlo ? dring[sm * B::FN + fi] : d0, dzp = zhi ? dring[sp * B::FN + fi] : d0;
        const float mzm = zlo ? mring[sm * B::FN + fi] : m0, mzp = zhi ? mring[sp * B::FN + fi] : m0;
        const Dr dr = demons_dr(d0, diff_scale(gx, nx), dp[fi + xh] - dp[fi + xl], mp[fi + xh] - mp[fi + xl],
                                diff_scale(gy, ny), dp[fi + yh] - dp[fi + yl], mp[fi + yh] - mp[fi + yl],
                                diff_scale(zo, nz), dzp - dzm, mzp - mzm, a.force_mode == DISC_FORCE_DOUBLE);
        const float drx = dr.x, dry = dr.y, drz = dr.z;
        const size_t g = (size_t)zo * plane + ooff[i];
        float rx, ry, rz;
        if (back == 1) {                       // staged in stage 1
          rx = ro[o];
          ry = ro[B::TN + o];
          rz = ro[2 * B::TN + o];
        } else {                               // last plane of the volume only
          rx = ldg_in(a.r, g, 3LL * N);
          ry = ldg_in(a.r, (long long)N + g, 3LL * N);
          rz = ldg_in(a.r, 2LL * N + g, 3LL * N);
        }
        const float keep = a.u_is_dr ? 0.0f : 1.0f;   // u = r + dr, or dr alone
        st_in(a.out, g, 3LL * N, fmaf(keep, rx, drx));
        st_in(a.out, (long long)N + g, 3LL * N, fmaf(keep, ry, dry));
        st_in(a.out, 2LL * N + g, 3LL * N, fmaf(keep, rz, drz));
        const bool nin = a.norm_hi <= a.norm_lo || (zo >= a.norm_lo && zo < a.norm_hi);   // the plane enters the norm sums
        acc0 += nin ? norm3(drx, dry, drz) : 0.0f;
        acc1 += nin ? norm3(rx, ry, rz) : 0.0f;
      }
    }
    }
    // the next step's stage 1 rewrites the staged planes (mring, zsf, ro) and the
    // next stage 2b the d ring: everything read above must be consumed first
    __syncthreads();
  }

  if (MODE == kModeIterate || MODE == kModeSsdLoss || MODE == kModeSsdAdjoint) {
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
      float t0 = 0.0f, t1 = 0.0f;
      for (int w = 0; w < kThreads / 32; ++w) {
        t0 += red[0][w];
        t1 += red[1][w];
      }
      a.partials[2 * part] = t0;
      a.partials[2 * part + 1] = t1;
    }
    __syncthreads();   // red[] is reused by the next body a persistent CTA runs
  }
}

template <int MODE, int H>
__global__ void __launch_bounds__(kThreads, 3) k_box_h(BoxArgs a) {
  const size_t part = (size_t)blockIdx.x + (size_t)gridDim.x * (blockIdx.y + (size_t)gridDim.y * blockIdx.z);
  box_body<MODE, H>(a, blockIdx.x, blockIdx.y, blockIdx.z, part);
}

// Batched launch over the work table of many volumes: work item i belongs to the
// volume p with offset[p] <= i < offset[p + 1] and is that volume's CTA
// i - offset[p] in x-fastest order of its own grid.  With persistent = 1 the
// grid is smaller than the table and each CTA strides over it.
template <int MODE, int H>
__global__ void __launch_bounds__(kThreads, 3) k_box_h_batch(const __grid_constant__ BoxBatch bt) {
  const int total = bt.offset[bt.count];
  for (int i = blockIdx.x; i < total; i += gridDim.x) {
    int p = 0;
    while (p + 1 < bt.count && bt.offset[p + 1] <= i) ++p;
    const int j = i - bt.offset[p];
    const dim3 g = bt.grid[p];
    const int bx = j % g.x, by = (j / g.x) % g.y, bz = j / (g.x * g.y);
    box_body<MODE, H>(bt.args[p], bx, by, bz, (size_t)j);
  }
}

constexpr int kMaxDevices = 64;

template <int MODE, int H>
cudaError_t launch_fast(const BoxArgs& a, const BoxPlan& p, cudaStream_t s) {
  static int set[kMaxDevices] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  if (!set[dev]) {
    e = cudaFuncSetAttribute(k_box_h<MODE, H>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)FastLayout<MODE, H>::bytes);
    if (e != cudaSuccess) return e;
    // prefer the largest shared-memory carveout so that several CTAs fit per SM
    e = cudaFuncSetAttribute(k_box_h<MODE, H>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    set[dev] = 1;
  }
  k_box_h<MODE, H><<<p.grid, kThreads, p.smem, s>>>(a);
  return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_fast_h(const BoxArgs& a, const BoxPlan& p, cudaStream_t s) {
  switch (a.hx) {
    case 1: return launch_fast<MODE, 1>(a, p, s);
    case 2: return launch_fast<MODE, 2>(a, p, s);
    case 3: return launch_fast<MODE, 3>(a, p, s);
    case 4: return launch_fast<MODE, 4>(a, p, s);
    case 5: return launch_fast<MODE, 5>(a, p, s);
    case 6: return launch_fast<MODE, 6>(a, p, s);
    case 7: return launch_fast<MODE, 7>(a, p, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int MODE, int H>
int occ_one(size_t smem) {
  // the opt-in shared memory size and carveout change the answer: set them first
  if (cudaFuncSetAttribute(k_box_h<MODE, H>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess ||
      cudaFuncSetAttribute(k_box_h<MODE, H>, cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_box_h<MODE, H>, kThreads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return n < 1 ? 1 : n;
}

template <int MODE>
int fast_occ(int h, size_t smem) {
  switch (h) {
    case 1: return occ_one<MODE, 1>(smem);
    case 2: return occ_one<MODE, 2>(smem);
    case 3: return occ_one<MODE, 3>(smem);
    case 4: return occ_one<MODE, 4>(smem);
    case 5: return occ_one<MODE, 5>(smem);
    case 6: return occ_one<MODE, 6>(smem);
    case 7: return occ_one<MODE, 7>(smem);
    default: return 1;
  }
}

template <int MODE>
size_t fast_bytes(int h) {
  switch (h) {
    case 1: return FastLayout<MODE, 1>::bytes;
    case 2: return FastLayout<MODE, 2>::bytes;
    case 3: return FastLayout<MODE, 3>::bytes;
    case 4: return FastLayout<MODE, 4>::bytes;
    case 5: return FastLayout<MODE, 5>::bytes;
    case 6: return FastLayout<MODE, 6>::bytes;
    case 7: return FastLayout<MODE, 7>::bytes;
    default: return 0;
  }
}

}  // namespace

bool box_fast_ok(int nx, int ny, int nz, int hx, int hy, int hz) {
  return hx == hy && hy == hz && hx >= 1 && hx <= 7 && (double)nx * ny * nz * 3.0 < 2147483647.0;
}

size_t box_fast_smem(int mode, int h) {
  switch (mode) {
    case kModeStatic: return fast_bytes<kModeStatic>(h);
    case kModeIterate: return fast_bytes<kModeIterate>(h);
    case kModeCorrected: return fast_bytes<kModeCorrected>(h);
    case kModeSsdLoss: return fast_bytes<kModeSsdLoss>(h);
    case kModeSsdAdjoint: return fast_bytes<kModeSsdAdjoint>(h);
    case kModeMaskAB: return fast_bytes<kModeMaskAB>(h);
    default: return 0;
  }
}

cudaError_t box_fast_launch_batch(const BoxBatch& bt, int h, int total, int grid, size_t smem,
                                  cudaStream_t s) {
  if (grid < 1) return cudaSuccess;
  switch (h) {
#define BCASE(HH)                                                                                   \
  case HH: {                                                                                        \
    static int set[kMaxDevices] = {};                                                              \
    int dev = 0;                                                                                    \
    cudaError_t e = cudaGetDevice(&dev);                                                            \
    if (e != cudaSuccess) return e;                                                                 \
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;                               \
    if (!set[dev]) {                                                                                \
      e = cudaFuncSetAttribute(k_box_h_batch<kModeIterate, HH>,                                     \
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);            \
      if (e != cudaSuccess) return e;                                                               \
      e = cudaFuncSetAttribute(k_box_h_batch<kModeIterate, HH>,                                     \
                               cudaFuncAttributePreferredSharedMemoryCarveout,                      \
                               (int)cudaSharedmemCarveoutMaxShared);                                \
      if (e != cudaSuccess) return e;                                                               \
      set[dev] = 1;                                                                                 \
    }                                                                                               \
    k_box_h_batch<kModeIterate, HH><<<grid, kThreads, smem, s>>>(bt);                               \
    return cudaGetLastError();                                                                      \
  }
    BCASE(1) BCASE(2) BCASE(3) BCASE(4) BCASE(5) BCASE(6) BCASE(7)
#undef BCASE
    default: return cudaErrorInvalidValue;
  }
  (void)total;
}

int box_fast_occupancy(int mode, int h, size_t smem) {
  switch (mode) {
    case kModeStatic: return fast_occ<kModeStatic>(h, smem);
    case kModeIterate: return fast_occ<kModeIterate>(h, smem);
    case kModeCorrected: return fast_occ<kModeCorrected>(h, smem);
    case kModeSsdLoss: return fast_occ<kModeSsdLoss>(h, smem);
    case kModeSsdAdjoint: return fast_occ<kModeSsdAdjoint>(h, smem);
    case kModeMaskAB: return fast_occ<kModeMaskAB>(h, smem);
    default: return 1;
  }
}

cudaError_t box_fast_launch(int mode, const BoxArgs& a, const BoxPlan& p, cudaStream_t s) {
  switch (mode) {
    case kModeStatic: return launch_fast_h<kModeStatic>(a, p, s);
    case kModeIterate: return launch_fast_h<kModeIterate>(a, p, s);
    case kModeCorrected: return launch_fast_h<kModeCorrected>(a, p, s);
    case kModeSsdLoss: return launch_fast_h<kModeSsdLoss>(a, p, s);
    case kModeSsdAdjoint: return launch_fast_h<kModeSsdAdjoint>(a, p, s);
    case kModeMaskAB: return launch_fast_h<kModeMaskAB>(a, p, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace disc
