// Patch-moment pass fed by the Tensor Memory Accelerator (sm_103a).
//
// The arithmetic is that of the cubic-patch kernels of box_fast.cu: exact
// integer sliding sums of q = rint(v 2^e) and q^2 over the truncated patch
// (Eq. 3), the patch moments (Appendix A.4), the moment-matched CBCT kept as
// d = I'_s - m (Eqs. 5-6) and, in iteration mode, the demons force of Eq. (1)
// with grad I'_s = grad d + grad m and the update u = r + dr (Algorithm A1
// steps 3-5).  What differs is how the z march is fed: every global read is a
// bulk tensor copy (cp.async.bulk.tensor) into shared memory, issued by one
// thread and completed on an mbarrier, one plane ahead of its use:
//   group A, issued once the entering plane of step z has been summed:
//     the W box (patch halo) of the entering plane z + 1, the W box of the
//     plane that leaves the window, and the F box of m at the next centre plane;
//   group B, issued at the top of step z and awaited after the x sums:
//     the F box of zs at the centre plane and the r tile of the force plane.
// The first planes of the window, which only enter the z sums, come as bursts of
// W boxes staged over the buffers the march has not used yet (one wait per
// burst, not per plane).
// Out-of-volume parts of a box arrive as zeros, which is exactly what the
// truncated sums need, so the march has no per-element bounds tests and no
// per-thread global loads.  A box starts on a 16-byte boundary in x (x offsets
// are multiples of 4 floats), so the W and F boxes are a few columns wider than
// the halo needs.  Every wait is bounded: after about a second without
// completion the CTA raises the error word, waits (bounded again) for its own
// copies and returns.

#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdlib>
#include <mutex>

#include "box_dev.cuh"
#include "internal.cuh"
#include "tma_dev.cuh"

namespace disc {

namespace {

// Error word of launches that were given none (kernel-level entry points).
__device__ int g_box_err;


template <int MODE, int H>
struct TmaLayout {
  static constexpr int EXT = (MODE == kModeIterate) ? 1 : 0;   // gradient halo of the force
  static constexpr int TX = 32, TY = 16;
  static constexpr int FX = TX + 2 * EXT, FY = TY + 2 * EXT;    // moment (F) region
  static constexpr int WX = FX + 2 * H, WY = FY + 2 * H;        // patch-sum (W) region
  static constexpr int WXP = WX | 1;                            // odd row stride of the z sums
  static constexpr int WN = WX * WY;
  static constexpr int K1 = (WN + kThreads - 1) / kThreads;     // W columns per thread
  static constexpr int XW = ceil4(EXT + H);                     // W box: x from x0 - XW,
  static constexpr int WXT = ceil4(XW + TX + EXT + H);          //   WXT floats wide, WY rows
  static constexpr int WOFF = XW - EXT - H;                     // column of W element 0 in the box
  static constexpr int XF = ceil4(EXT);                         // F box: x from x0 - XF,
  static constexpr int FXT = ceil4(XF + TX + EXT);              //   FXT floats wide, FY rows
  static constexpr int FO = XF - EXT;                           // column of F element 0 in the box
  static constexpr int FN = FXT * FY;                           // floats of an F plane
  static constexpr int NMS = EXT ? 4 : 2;                       // F planes of m in flight
  static constexpr int TN = TX * TY;
  static constexpr int KO = TN / kThreads;                      // tile voxels per thread
  static_assert(TN % kThreads == 0 && kThreads % TX == 0, "tile and CTA shape");
  // about half as many x tasks as threads: longer slides amortise the initial window
  static constexpr int NSX0 = (kThreads / 2 / WY) < 1 ? 1 : (kThreads / 2 / WY);
  static constexpr int SX = (FX + NSX0 - 1) / NSX0;             // x outputs per sliding task
  static constexpr int NSX = (FX + SX - 1) / SX;
  static constexpr int NSY0 = (kThreads / FX) < 1 ? 1 : (kThreads / FX);
  static constexpr int SY = (FY + NSY0 - 1) / NSY0;             // y outputs per sliding task
  static constexpr int NSY = (FY + SY - 1) / SY;
  static constexpr int NP = (2 * H + 1) * (2 * H + 1) * (2 * H + 1);
  static constexpr uint32_t WB = 4u * WXT * WY;                 // bytes of a W box
  static constexpr uint32_t FB = 4u * FXT * FY;                 // bytes of an F box
  static constexpr uint32_t RB = 12u * TN;                      // bytes of the r tile
  static constexpr int MS = (int)(al128(FB) / 4);               // float stride of the m planes
  // shared memory map; the TMA destinations come first, on 128-byte boundaries
  static constexpr size_t o_wn = 0;                             // W box, entering plane
  static constexpr size_t o_wo = o_wn + al128(WB);              // W box, leaving plane
  static constexpr size_t o_mr = o_wo + al128(WB);              // NMS F planes of m
  static constexpr size_t o_zs = o_mr + NMS * al128(FB);        // F plane of zs
  static constexpr size_t o_ro = o_zs + (MODE == kModeStatic ? 0 : al128(FB));   // r tile [3][TY][TX]
  static constexpr size_t o_s2z = o_ro + (EXT ? al128(RB) : 0); // z sums of q^2 (int64)
  static constexpr size_t o_xb1 = o_s2z + 8 * (size_t)WY * WXP; // x sums of q
  static constexpr size_t o_xb2 = o_xb1 + 8 * (size_t)WY * FX;  // x sums of q^2
  static constexpr size_t o_s1z = o_xb2 + 8 * (size_t)WY * FX;  // z sums of q (int32)
  static constexpr size_t o_dr = o_s1z + 4 * (size_t)WY * WXP;  // 3 F planes of d
  static constexpr size_t o_red = o_dr + (EXT ? 12 * (size_t)FN : 0);   // norm partials
  static constexpr size_t o_bar = (o_red + 8 * (kThreads / 32) + 7) & ~(size_t)7;   // 2 mbarriers
  static constexpr size_t bytes = o_bar + 16;
  // W boxes the warm-up burst stages at once, over every buffer below o_red
  static constexpr int WST = (int)(o_red / al128(WB));
  static_assert(WST >= 2, "staging area");
};

// Step bookkeeping shared by every thread (all values are CTA-uniform).
struct March {
  int z0, z1, zc_lo, zc_hi, zi0, zi1, nz;
};

template <int MODE, int H>
__device__ __forceinline__ uint32_t bytes_a(const March& s, int zi) {
  using B = TmaLayout<MODE, H>;
  const int zc = zi - H;
  return (zi < s.nz ? B::WB : 0u) + (zi - (2 * H + 1) >= s.zi0 ? B::WB : 0u) +
         (zc >= s.zc_lo && zc <= s.zc_hi ? B::FB : 0u);
}

template <int MODE, int H>
__device__ __forceinline__ uint32_t bytes_b(const March& s, int zi) {
  using B = TmaLayout<MODE, H>;
  const int zc = zi - H, zf = zc - 1;
  const bool do2 = zc >= s.zc_lo && zc <= s.zc_hi;
  const bool do3 = MODE == kModeIterate && zf >= s.z0 && zf < s.z1;
  return (do2 && MODE != kModeStatic ? B::FB : 0u) + (do3 ? B::RB : 0u);
}

// The CTA body: tile (bx, by), z chunk bz of the volume described by `a`;
// `part` indexes this CTA's norm partials.  The two mbarriers at B::o_bar are
// initialised by the kernel; pa and pb are their phase parities, carried over
// the bodies a persistent CTA runs (every phase armed in a body is awaited in
// it).  Returns false when a copy wait gave up: the CTA must stop.
template <int MODE, int H>
__device__ __forceinline__ bool box_tma_body(const BoxArgs& a, int bx, int by, int bz, size_t part,
                                             const CUtensorMap* map_w, const CUtensorMap* map_f,
                                             const CUtensorMap* map_z, const CUtensorMap* map_r,
                                             unsigned char* smem, uint32_t& pa, uint32_t& pb) {
  using B = TmaLayout<MODE, H>;
  if (a.stop != nullptr && *(volatile const int*)a.stop != 0) return true;
  int* err = a.err ? a.err : &g_box_err;
  float* wn = reinterpret_cast<float*>(smem + B::o_wn);
  float* wo = reinterpret_cast<float*>(smem + B::o_wo);
  float* mring = reinterpret_cast<float*>(smem + B::o_mr);
  float* zsf = reinterpret_cast<float*>(smem + B::o_zs);
  float* ro = reinterpret_cast<float*>(smem + B::o_ro);
  long long* s2z = reinterpret_cast<long long*>(smem + B::o_s2z);
  long long* xb1 = reinterpret_cast<long long*>(smem + B::o_xb1);
  long long* xb2 = reinterpret_cast<long long*>(smem + B::o_xb2);
  int* s1z = reinterpret_cast<int*>(smem + B::o_s1z);
  float* dring = reinterpret_cast<float*>(smem + B::o_dr);
  float* red = reinterpret_cast<float*>(smem + B::o_red);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + B::o_bar);   // [0] group A, [1] group B

  const int tid = threadIdx.x;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int plane = nx * ny;                  // 3 N < 2^31 is checked on the host
  const int N = plane * nz;
  const int x0 = bx * B::TX, y0 = by * B::TY;
  March st;
  st.nz = nz;
  st.z0 = bz * a.zlen;
  st.z1 = min(nz, st.z0 + a.zlen);
  st.zc_lo = max(0, st.z0 - B::EXT);
  st.zc_hi = min(nz - 1, st.z1 - 1 + B::EXT);
  st.zi0 = max(0, st.zc_lo - H);
  // iteration mode: the force of plane zf is computed in the step whose centre
  // plane is zf + 1, so the march runs to centre plane z1 (a step without
  // moments when z1 = nz)
  st.zi1 = (MODE == kModeIterate ? st.z1 : st.zc_hi) + H;
  const int z0 = st.z0, z1 = st.z1;
  const float qs = a.qscale, inv_qs = a.inv_qscale, vfl = a.var_floor;

  auto issue_a = [&](int zi) {               // thread 0 only
    const uint32_t nb = bytes_a<MODE, H>(st, zi);
    if (nb == 0) return;
    mbar_expect_tx(&bar[0], zi == st.zi0 ? nb + a.stall_tx : nb);
    const int zo = zi - (2 * H + 1), zc = zi - H;
    if (zi < nz) tma_load_3d(wn, map_w, x0 - B::XW, y0 - B::EXT - H, zi, &bar[0]);
    if (zo >= st.zi0) tma_load_3d(wo, map_w, x0 - B::XW, y0 - B::EXT - H, zo, &bar[0]);
    if (zc >= st.zc_lo && zc <= st.zc_hi)
      tma_load_3d(mring + ((unsigned)zc % B::NMS) * B::MS, map_f, x0 - B::XF, y0 - B::EXT, zc, &bar[0]);
  };
  auto issue_b = [&](int zi) {               // thread 0 only
    const uint32_t nb = bytes_b<MODE, H>(st, zi);
    if (nb == 0) return;
    mbar_expect_tx(&bar[1], nb);
    const int zc = zi - H, zf = zc - 1;
    const bool do2 = zc >= st.zc_lo && zc <= st.zc_hi;
    const bool do3 = MODE == kModeIterate && zf >= st.z0 && zf < st.z1;
    if (MODE != kModeStatic && do2) tma_load_3d(zsf, map_z, x0 - B::XF, y0 - B::EXT, zc, &bar[1]);
    if (do3) tma_load_4d(ro, map_r, x0, y0, zf, 0, &bar[1]);
  };

  // ---- per-thread maps, fixed for the whole march ------------------------------
  int stg[B::K1], sidx[B::K1], s1r[B::K1];   // W box index, z-sum index, running z sums
  long long s2r[B::K1];
#pragma unroll
  for (int k = 0; k < B::K1; ++k) {
    const int e = tid + k * kThreads;
    const int wy = e / B::WX, wx = e - wy * B::WX;
    sidx[k] = e < B::WN ? wy * B::WXP + wx : -1;
    stg[k] = wy * B::WXT + wx + B::WOFF;
    s1r[k] = 0;
    s2r[k] = 0;
  }
  // force stage: tile voxel (ox, oy_i); one-sided differences at the faces are
  // s * (v[+r] - v[-l]) with offsets l, r in {0, 1} and s in {0, 1/2, 1}
  const int ox = tid % B::TX;
  const int gxo = x0 + ox;
  const int lxo = gxo > 0 ? -1 : 0, rxo = gxo < nx - 1 ? 1 : 0;
  const float sxo = (lxo != 0 && rxo != 0) ? 0.5f : ((lxo != 0 || rxo != 0) ? 1.0f : 0.0f);
  int fo3[B::KO], goff3[B::KO], lyo[B::KO], ryo[B::KO];
  float syo[B::KO];
#pragma unroll
  for (int i = 0; i < B::KO; ++i) {
    const int oy = tid / B::TX + i * (kThreads / B::TX);
    const int gy = y0 + oy;
    const bool ok = gxo < nx && gy < ny;
    fo3[i] = ok ? (oy + B::EXT) * B::FXT + ox + B::EXT + B::FO : -1;
    goff3[i] = gy * nx + gxo;
    lyo[i] = gy > 0 ? -B::FXT : 0;
    ryo[i] = gy < ny - 1 ? B::FXT : 0;
    syo[i] = (lyo[i] != 0 && ryo[i] != 0) ? 0.5f : ((lyo[i] != 0 || ryo[i] != 0) ? 1.0f : 0.0f);
  }

  float acc0 = 0.0f, acc1 = 0.0f;
  const float keep = a.u_is_dr ? 0.0f : 1.0f;   // the force stage writes u = keep r + dr

  // ---- warm-up: planes zi0 .. zw - 1 only enter the z sums (no plane leaves the
  // window and no centre plane is due), so they arrive as bursts of W boxes in the
  // buffers the march has not yet used, one copy wait per burst instead of one per
  // plane, and are summed in the order the march would have summed them
  const int zw = st.zc_lo + H;              // first step with a centre plane
  {
    fence_proxy_async();                    // earlier generic writes of the staging area
    __syncthreads();
    const int zb_end = min(zw, nz);
    for (int zb = st.zi0; zb < zb_end; zb += B::WST) {
      const int nb = min(B::WST, zb_end - zb);
      if (tid == 0) {
        mbar_expect_tx(&bar[0], (uint32_t)nb * B::WB + (zb == st.zi0 ? a.stall_tx : 0u));
        for (int j = 0; j < nb; ++j)
          tma_load_3d(smem + j * al128(B::WB), map_w, x0 - B::XW, y0 - B::EXT - H, zb + j, &bar[0]);
      }
      int bad = 0;
      if (tid == 0) bad = !mbar_wait(&bar[0], pa);
      if (__syncthreads_or(bad)) {
        if (tid == 0) {
          atomicOr(err, 1);
          mbar_wait(&bar[0], pa);          // bounded: let this CTA's copies drain
        }
        __syncthreads();
        return false;
      }
      pa ^= 1u;
      for (int j = 0; j < nb; ++j) {
        const float* wj = reinterpret_cast<const float*>(smem + j * al128(B::WB));
#pragma unroll
        for (int k = 0; k < B::K1; ++k) {
          if (sidx[k] < 0) continue;
          const int qn = __float2int_rn(wj[stg[k]] * qs);
          s1r[k] += qn;
          s2r[k] += (long long)qn * qn;
        }
      }
      __syncthreads();                       // the staging area is consumed
    }
  }
  if (tid == 0) issue_a(zw);

  // slot of the centre plane in the ring of d planes, kept incrementally
  int zc3 = ((zw - H) % 3 + 3) % 3;
  for (int zi = zw; zi <= st.zi1; ++zi, zc3 = (zc3 == 2 ? 0 : zc3 + 1)) {
    const int zc = zi - H;                   // centre plane of the patch window
    const bool do2 = zc >= st.zc_lo && zc <= st.zc_hi;
    const int zf = zc - 1;                   // plane whose force is computed this step
    const bool do3 = MODE == kModeIterate && zf >= z0 && zf < z1;
    // ---- top of the step: group A of this step has landed -----------------------
    {
      int bad = 0;
      const bool armed = bytes_a<MODE, H>(st, zi) != 0;
      if (armed && tid == 0) bad = !mbar_wait(&bar[0], pa);
      if (__syncthreads_or(bad)) {
        if (tid == 0) {
          atomicOr(err, 1);
          mbar_wait(&bar[0], pa);            // bounded: let this CTA's copies drain
        }
        __syncthreads();
        return false;
      }
      if (armed) pa ^= 1u;
    }
    const uint32_t nbb = bytes_b<MODE, H>(st, zi);
    if (tid == 0) issue_b(zi);

    // ---- stage 1: z sliding sums of the W columns from the staged boxes ---------
    const bool has_new = zi < nz, has_old = zi - (2 * H + 1) >= st.zi0;
#pragma unroll
    for (int k = 0; k < B::K1; ++k) {
      if (sidx[k] < 0) continue;
      const float vn = has_new ? wn[stg[k]] : 0.0f;
      const float vo = has_old ? wo[stg[k]] : 0.0f;
      const int qn = __float2int_rn(vn * qs), qo = __float2int_rn(vo * qs);
      s1r[k] += qn - qo;
      s2r[k] += (long long)qn * qn - (long long)qo * qo;
      s1z[sidx[k]] = s1r[k];
      s2z[sidx[k]] = s2r[k];
    }
    __syncthreads();
    if (tid == 0 && zi < st.zi1) issue_a(zi + 1);   // the W boxes are consumed
    if (!do2 && !do3) continue;              // uniform; group B was not armed

    // ---- stage 2a: x window sums, sliding, one task per (segment, row) ---------
    for (int t = do2 ? tid : B::NSX * B::WY; t < B::NSX * B::WY; t += kThreads) {
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
    {
      int bad = 0;
      if (nbb != 0 && tid == 0) bad = !mbar_wait(&bar[1], pb);
      if (__syncthreads_or(bad)) {
        if (tid == 0) {
          atomicOr(err, 1);
          mbar_wait(&bar[1], pb);
          if (zi < st.zi1 && bytes_a<MODE, H>(st, zi + 1) != 0) mbar_wait(&bar[0], pa);
        }
        __syncthreads();
        return false;
      }
      if (nbb != 0) pb ^= 1u;
    }

    // ---- stage 2b: y window sums, sliding; moments and correction --------------
    const bool zin = zc >= H && zc < nz - H;
    const int nzc = box_count(zc, nz, H);
    const bool out_plane = zc >= z0 && zc < z1;
    const float* mr = mring + ((unsigned)zc % B::NMS) * B::MS;
    float* dcur = dring + zc3 * B::FN;
    for (int t = do2 ? tid : B::NSY * B::FX; t < B::NSY * B::FX; t += kThreads) {
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
        const int fi = fy * B::FXT + fx + B::FO;
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
          dcur[fi] = d;
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
    if (do3) {
      __syncthreads();
      // ---- stage 3: demons force (Eq. 1) and update of plane zf = zc - 1 -------
      const int zo = zf;
      const bool zlo = zo > 0, zhi = zo < nz - 1;
      const float sz = (zlo && zhi) ? 0.5f : ((zlo || zhi) ? 1.0f : 0.0f);
      const int s_m1 = zc3 == 2 ? 0 : zc3 + 1;      // slot of zc - 2
      const int s_0 = zc3 == 0 ? 2 : zc3 - 1;       // slot of zc - 1 = zo
      const float* dp = dring + s_0 * B::FN;
      const float* dzm = dring + (zlo ? s_m1 : s_0) * B::FN;
      const float* dzp = dring + (zhi ? zc3 : s_0) * B::FN;
      const float* mp = mring + ((unsigned)zo % B::NMS) * B::MS;
      const float* mzm = mring + ((unsigned)(zlo ? zo - 1 : zo) % B::NMS) * B::MS;
      const float* mzp = mring + ((unsigned)(zhi ? zo + 1 : zo) % B::NMS) * B::MS;
      const bool nin = a.norm_hi <= a.norm_lo || (zo >= a.norm_lo && zo < a.norm_hi);   // the plane enters the norm sums
      float* out0 = a.out + (size_t)zo * plane;
#pragma unroll
      for (int i = 0; i < B::KO; ++i) {
        const int fi = fo3[i];
        if (fi < 0) continue;
        const Dr dr = demons_dr(dp[fi], sxo, dp[fi + rxo] - dp[fi + lxo], mp[fi + rxo] - mp[fi + lxo], syo[i],
                                dp[fi + ryo[i]] - dp[fi + lyo[i]], mp[fi + ryo[i]] - mp[fi + lyo[i]], sz,
                                dzp[fi] - dzm[fi], mzp[fi] - mzm[fi], a.force_mode == DISC_FORCE_DOUBLE);
        const int o = tid + i * kThreads;
        const float rx = ro[o], ry = ro[B::TN + o], rz = ro[2 * B::TN + o];   // staged by group B
        float* po = out0 + goff3[i];
        st_at(po, a.out, 3LL * N, fmaf(keep, rx, dr.x));
        st_at(po + N, a.out, 3LL * N, fmaf(keep, ry, dr.y));
        st_at(po + 2 * (size_t)N, a.out, 3LL * N, fmaf(keep, rz, dr.z));
        acc0 += nin ? norm3(dr.x, dr.y, dr.z) : 0.0f;
        acc1 += nin ? norm3(rx, ry, rz) : 0.0f;
      }
    }
    // the next step's stage 1 rewrites the z sums, group B the zs and r slots,
    // and the next stage 2b a d plane that stage 3 may still read: its top
    // barrier separates them
  }

  if (MODE == kModeIterate || MODE == kModeSsdLoss || MODE == kModeSsdAdjoint) {
    for (int off = 16; off > 0; off >>= 1) {
      acc0 += __shfl_down_sync(0xffffffffu, acc0, off);
      acc1 += __shfl_down_sync(0xffffffffu, acc1, off);
    }
    const int lane = tid & 31, wid = tid >> 5;
    if (lane == 0) {
      red[wid] = acc0;
      red[kThreads / 32 + wid] = acc1;
    }
    __syncthreads();
    if (tid == 0 && a.partials != nullptr) {
      float t0 = 0.0f, t1 = 0.0f;
      for (int w = 0; w < kThreads / 32; ++w) {
        t0 += red[w];
        t1 += red[kThreads / 32 + w];
      }
      a.partials[2 * part] = t0;
      a.partials[2 * part + 1] = t1;
    }
  }
  return true;
}

// Shared-memory base check (TMA destinations need 128-byte alignment) and
// barrier set-up, once per CTA.
template <int MODE, int H>
__device__ __forceinline__ bool tma_cta_setup(unsigned char* smem, int* err) {
  using B = TmaLayout<MODE, H>;
  if ((smem_addr(smem) & 127u) != 0u) {
    if (threadIdx.x == 0) atomicOr(err ? err : &g_box_err, 2);
    return false;
  }
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + B::o_bar);
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_proxy_async();
  }
  __syncthreads();
  return true;
}

template <int MODE, int H>
__global__ void __launch_bounds__(kThreads, 3)
    k_box_tma(const BoxArgs a, const __grid_constant__ CUtensorMap map_w, const __grid_constant__ CUtensorMap map_f,
              const __grid_constant__ CUtensorMap map_z, const __grid_constant__ CUtensorMap map_r) {
  extern __shared__ __align__(128) unsigned char smem[];
  pdl_wait();
  pdl_release();
  if (a.stop != nullptr && *(volatile const int*)a.stop != 0) return;
  if (!tma_cta_setup<MODE, H>(smem, a.err)) return;
  uint32_t pa = 0, pb = 0;
  const size_t part = (size_t)blockIdx.x + (size_t)gridDim.x * (blockIdx.y + (size_t)gridDim.y * blockIdx.z);
  box_tma_body<MODE, H>(a, blockIdx.x, blockIdx.y, blockIdx.z, part, &map_w, &map_f, &map_z, &map_r, smem, pa,
                        pb);
}

// Batched launch over the work table of many volumes (as k_box_h_batch): work
// item i belongs to volume p with offset[p] <= i < offset[p + 1].  The tensor
// maps of volume p are maps[4p .. 4p + 3] (W box, F box of m, F box of zs, r
// tile) in global memory, written by the host before the launch.
template <int MODE, int H>
__global__ void __launch_bounds__(kThreads, 3)
    k_box_tma_batch(const __grid_constant__ BoxBatch bt, const CUtensorMap* __restrict__ maps) {
  extern __shared__ __align__(128) unsigned char smem[];
  pdl_wait();
  pdl_release();
  if (!tma_cta_setup<MODE, H>(smem, nullptr)) return;
  uint32_t pa = 0, pb = 0;
  const int total = bt.offset[bt.count];
  for (int i = blockIdx.x; i < total; i += gridDim.x) {
    int p = 0;
    while (p + 1 < bt.count && bt.offset[p + 1] <= i) ++p;
    const int j = i - bt.offset[p];
    const dim3 g = bt.grid[p];
    const int bx = j % g.x, by = (j / g.x) % g.y, bz = j / (g.x * g.y);
    const CUtensorMap* m = maps + 4 * p;
    if (threadIdx.x == 0) {
      // the maps reach the tensor-map proxy through global memory
      for (int k = 0; k < 4; ++k)
        asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                         reinterpret_cast<uint64_t>(m + k))
                     : "memory");
    }
    __syncthreads();   // the previous body's last reads of the staging buffers are done
    if (!box_tma_body<MODE, H>(bt.args[p], bx, by, bz, (size_t)j, m, m + 1, m + 2, m + 3, smem, pa, pb)) return;
  }
}

// ---- host side ---------------------------------------------------------------
bool encode(CUtensorMap* m, const float* base, int rank, int nx, int ny, int nz, uint32_t bx, uint32_t by,
            uint32_t bc) {
  return tma_encode_volume(m, base, rank, nx, ny, nz, bx, by, bc);
}

constexpr int kMaxDevices = 64;

// The four tensor maps of a volume: W box of src, F box of src, F box of zs, r tile.
template <int MODE, int H>
bool encode_maps(const BoxArgs& a, CUtensorMap* m) {
  using B = TmaLayout<MODE, H>;
  for (int k = 0; k < 4; ++k) m[k] = CUtensorMap{};
  if (!encode(&m[0], a.src, 3, a.nx, a.ny, a.nz, B::WXT, B::WY, 1) ||
      !encode(&m[1], a.src, 3, a.nx, a.ny, a.nz, B::FXT, B::FY, 1))
    return false;
  if (MODE != kModeStatic && !encode(&m[2], a.zs, 3, a.nx, a.ny, a.nz, B::FXT, B::FY, 1)) return false;
  if (MODE == kModeIterate && !encode(&m[3], a.r, 4, a.nx, a.ny, a.nz, B::TX, B::TY, 3)) return false;
  return true;
}

// Opt-in shared memory and the shared-memory carveout, once per device and kernel.
template <typename K>
cudaError_t prepare(K kernel, size_t smem, int* set) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  if (set[dev]) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  set[dev] = 1;
  return cudaSuccess;
}

template <int MODE, int H>
cudaError_t launch_tma(const BoxArgs& a, const BoxPlan& p, cudaStream_t s) {
  using B = TmaLayout<MODE, H>;
  static int set[kMaxDevices] = {};
  CUtensorMap m[4];
  if (!encode_maps<MODE, H>(a, m)) return cudaErrorInvalidValue;
  cudaError_t e = prepare(k_box_tma<MODE, H>, B::bytes, set);
  if (e != cudaSuccess) return e;
  BoxArgs b = a;
  // DISC_SW_TMA_STALL: the iteration pass waits for 16 bytes no copy delivers
  // (exercises the bounded wait and the timeout report; nothing else changes)
  b.stall_tx = (MODE == kModeIterate && (test_switches() & DISC_SW_TMA_STALL)) ? 16u : 0u;
  return launch_pdl(k_box_tma<MODE, H>, p.grid, dim3(kThreads), B::bytes, s, b, m[0], m[1], m[2], m[3]);
}

template <int MODE, int H>
cudaError_t launch_tma_batch(const BoxBatch* bt, const CUtensorMap* maps, int grid, cudaStream_t s) {
  using B = TmaLayout<MODE, H>;
  static int set[kMaxDevices] = {};
  cudaError_t e = prepare(k_box_tma_batch<MODE, H>, B::bytes, set);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_box_tma_batch<MODE, H>, dim3(grid), dim3(kThreads), B::bytes, s, *bt, maps);
}

template <typename K>
int occupancy(K kernel, size_t smem) {
  if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, kThreads, smem) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return n < 1 ? 1 : n;
}

template <int MODE, int H>
int occ_tma(size_t smem) {
  return occupancy(k_box_tma<MODE, H>, smem);
}

// Compile-time table over (mode, H): fn(mode, h) dispatches to F<MODE, H>.
template <template <int, int> class F, typename R, typename... Args>
R dispatch(int mode, int h, R fallback, Args... args) {
#define DISC_TMA_H(M)                                     \
  switch (h) {                                            \
    case 1: return F<M, 1>::run(args...);                 \
    case 2: return F<M, 2>::run(args...);                 \
    case 3: return F<M, 3>::run(args...);                 \
    case 4: return F<M, 4>::run(args...);                 \
    case 5: return F<M, 5>::run(args...);                 \
    case 6: return F<M, 6>::run(args...);                 \
    case 7: return F<M, 7>::run(args...);                 \
    default: return fallback;                             \
  }
  switch (mode) {
    case kModeStatic: DISC_TMA_H(kModeStatic)
    case kModeIterate: DISC_TMA_H(kModeIterate)
    case kModeCorrected: DISC_TMA_H(kModeCorrected)
    case kModeSsdLoss: DISC_TMA_H(kModeSsdLoss)
    case kModeSsdAdjoint: DISC_TMA_H(kModeSsdAdjoint)
    case kModeMaskAB: DISC_TMA_H(kModeMaskAB)
    default: return fallback;
  }
#undef DISC_TMA_H
}

template <int MODE, int H>
struct Bytes {
  static size_t run() { return TmaLayout<MODE, H>::bytes; }
};
template <int MODE, int H>
struct Occ {
  static int run(size_t smem) { return occ_tma<MODE, H>(smem); }
};
template <int MODE, int H>
struct Launch {
  static cudaError_t run(const BoxArgs* a, const BoxPlan* p, cudaStream_t s) { return launch_tma<MODE, H>(*a, *p, s); }
};
template <int MODE, int H>
struct Maps {
  static bool run(const BoxArgs* a, CUtensorMap* m) { return encode_maps<MODE, H>(*a, m); }
};
template <int MODE, int H>
struct LaunchBatch {   // iteration mode only
  static cudaError_t run(const BoxBatch* bt, const CUtensorMap* maps, int grid, cudaStream_t s) {
    return MODE == kModeIterate ? launch_tma_batch<kModeIterate, H>(bt, maps, grid, s) : cudaErrorInvalidValue;
  }
};
template <int MODE, int H>
struct OccBatch {
  static int run(size_t smem) { return occupancy(k_box_tma_batch<kModeIterate, H>, smem); }
};
template <int MODE, int H>
struct Extent {   // smallest volume extents that hold every TMA box of this kernel
  static int run(int axis) {
    using B = TmaLayout<MODE, H>;
    return axis == 0 ? B::WXT : B::WY;
  }
};

bool tma_disabled() { return (test_switches() & DISC_SW_NO_TMA) != 0u; }

}  // namespace

bool box_tma_ok(int mode, int nx, int ny, int nz, int hx, int hy, int hz) {
  if (tma_disabled() || !box_fast_ok(nx, ny, nz, hx, hy, hz)) return false;
  if (nx % 4 != 0) return false;             // row stride: a multiple of 16 bytes
  const int ex = dispatch<Extent, int>(mode, hx, 0, 0), ey = dispatch<Extent, int>(mode, hx, 0, 1);
  if (ex == 0 || nx < ex || ny < ey || nz < 1) return false;
  return tma_encode_available();
}

bool box_tma_aligned(int mode, const BoxArgs& a) {
  auto al = [](const void* p) { return ((uintptr_t)p & 15u) == 0; };
  if (!al(a.src)) return false;
  if (mode != kModeStatic && !al(a.zs)) return false;
  if (mode == kModeIterate && !al(a.r)) return false;
  return true;
}

size_t box_tma_smem(int mode, int h) { return dispatch<Bytes, size_t>(mode, h, (size_t)0); }

int box_tma_occupancy(int mode, int h, size_t smem) { return dispatch<Occ, int>(mode, h, 1, smem); }

cudaError_t box_tma_launch(int mode, const BoxArgs& a, const BoxPlan& p, cudaStream_t s) {
  return dispatch<Launch, cudaError_t>(mode, a.hx, cudaErrorInvalidValue, &a, &p, s);
}

bool box_tma_encode(int mode, const BoxArgs& a, void* maps) {
  return dispatch<Maps, bool>(mode, a.hx, false, &a, static_cast<CUtensorMap*>(maps));
}

int box_tma_batch_occupancy(int h, size_t smem) { return dispatch<OccBatch, int>(kModeIterate, h, 1, smem); }

cudaError_t box_tma_launch_batch(const BoxBatch& bt, const void* maps, int h, int grid, cudaStream_t s) {
  if (grid < 1) return cudaSuccess;
  return dispatch<LaunchBatch, cudaError_t>(kModeIterate, h, cudaErrorInvalidValue, &bt,
                                            static_cast<const CUtensorMap*>(maps), grid, s);
}

// ---- tensor-map encoding shared by the bulk-copy-fed kernels ---------------------
namespace {
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

}  // namespace

bool tma_encode_available() { return encode_fn() != nullptr; }

// Plane-wise float32 volume [nz][ny][nx] (rank 3) or field [3][nz][ny][nx] (rank 4).
bool tma_encode_volume(CUtensorMap* m, const float* base, int rank, int nx, int ny, int nz, uint32_t bx,
                       uint32_t by, uint32_t bc) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[4] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz, 3};
  const cuuint64_t strides[3] = {(cuuint64_t)nx * 4, (cuuint64_t)nx * ny * 4, (cuuint64_t)nx * ny * nz * 4};
  const cuuint32_t box[4] = {bx, by, 1, bc};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, const_cast<float*>(base), dims, strides,
            box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t box_tma_error(cudaStream_t s, int* flag) {
  int* dev = nullptr;
  cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&dev), g_box_err);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(flag, dev, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && *flag != 0) e = cudaMemsetAsync(dev, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

}  // namespace disc
