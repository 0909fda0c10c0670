// Moment, correction, force and update pass on wide tiles (cubic patches,
// sm_103a): the hot pass of every iteration on the large levels.  The same
// kernel in its adjoint mode computes the SSD form's coefficients (the patch
// moments, the loss and A, B, C, D at the tile's own voxels; no force stage),
// and in its mask mode the a, b and xi of Eqs. 5-7 of the masked correction.
//
// Same arithmetic as the other cubic-patch kernels (box_fast.cu, box_tma.cu),
// so the outputs are bit-identical: exact integer sliding sums of q = rint(v 2^e)
// and q^2 over the truncated patch (Eq. 3), the patch moments (Appendix A.4),
// the moment-matched CBCT kept as d = I'_s - m (Eqs. 5-6), the demons force of
// Eq. (1) with grad I'_s = grad d + grad m, and u = r + dr (Algorithm A1 steps
// 3-5).  What differs is the work per voxel:
//  - tiles of TX x TY = 32 x 32 columns (two CTAs of 256 threads per SM): the
//    patch halo of the z sums costs 1.9 summed columns per output voxel at
//    patch 11^3 (2.4 on 32 x 16 tiles) and the x sums 1.5 (1.9);
//  - only the patch-halo boxes of m travel by bulk tensor copy (the entering
//    plane, the leaving plane and the moment region of the centre plane, one
//    group per z step); zs and r, read once per voxel, are loaded straight into
//    registers at the top of the step that uses them, so their latency hides
//    behind the sums;
//  - the q^2 z sums advance by one 32 x 32 -> 64-bit multiply-add,
//    q_new^2 - q_old^2 = (q_new - q_old)(q_new + q_old);
//  - the z-sum and x-sum planes have odd row strides (no bank conflicts on the
//    column-wise 64-bit reads);
//  - each CTA marches a balanced share of all (tile, plane) pairs of the volume,
//    possibly two tiles in turn, so every CTA of the single wave ends together.
// Every wait on a copy is bounded: after about a second without completion the
// CTA raises the error word, waits (bounded again) for its own copies and
// returns.

#include <cuda.h>
#include <cudaTypedefs.h>

#include "box_dev.cuh"
#include "internal.cuh"
#include "tma_dev.cuh"

namespace disc {

namespace {

__device__ int g_wide_err;   // error word of launches that were given none

constexpr int kWideThreads = 256;

template <int H, int TX, int TY>
struct WideLayout {
  static constexpr int NT = kWideThreads;
  static constexpr int FX = TX + 2, FY = TY + 2;               // moment region: tile + gradient halo
  static constexpr int WX = FX + 2 * H, WY = FY + 2 * H;       // z-summed columns: + patch halo
  static constexpr int WXP = WX | 1;                           // odd row stride of the z sums
  static constexpr int XBS = FX | 1;                           // odd row stride of the x sums
  static constexpr int WN = WX * WY;
  static constexpr int K1 = (WN + NT - 1) / NT;                // z-summed columns per thread
  static constexpr int XW = ceil4(1 + H);                      // W box: x from x0 - XW,
  static constexpr int WXT = ceil4(XW + TX + 1 + H);           //   WXT floats wide, WY rows
  static constexpr int WOFF = XW - 1 - H;                      // column of W element 0 in the box
  static constexpr int XF = 4;                                 // F box: x from x0 - 4,
  static constexpr int FXT = ceil4(XF + TX + 1);               //   FXT floats wide, FY rows
  static constexpr int FO = XF - 1;                            // column of F element 0 in the box
  static constexpr int FN = FXT * FY;                          // floats of an F plane
  static constexpr int NMS = 4;                                // F planes of m in flight
  static constexpr int QX = TX / 4;                            // force stage: x quads per tile row
  static_assert(TX % 4 == 0 && NT == QX * TY, "force stage: one x quad of the tile per thread");
  static_assert(FXT % 4 == 0 && (1 + FO) % 4 == 0, "force stage: 16-byte aligned quads in the F planes");
  static constexpr int NSX0 = (NT / WY) < 1 ? 1 : (NT / WY);   // x tasks: segments per W row
  static constexpr int SX = (FX + NSX0 - 1) / NSX0;
  static constexpr int NSX = (FX + SX - 1) / SX;
  static constexpr int NSY0 = (NT / FX) < 1 ? 1 : (NT / FX);   // y tasks: segments per F column
  static constexpr int SY = (FY + NSY0 - 1) / NSY0;
  static constexpr int NSY = (FY + SY - 1) / SY;
  static constexpr int NP = (2 * H + 1) * (2 * H + 1) * (2 * H + 1);
  static constexpr uint32_t WB = 4u * WXT * WY;                // bytes of a W box
  static constexpr uint32_t FB = 4u * FXT * FY;                // bytes of an F box
  static constexpr int MS = (int)(al128(FB) / 4);              // float stride of the m planes
  // shared memory map; the bulk-copy destinations first, on 128-byte boundaries
  static constexpr size_t o_wn = 0;                            // W box, entering plane
  static constexpr size_t o_wo = o_wn + al128(WB);             // W box, leaving plane
  static constexpr size_t o_mr = o_wo + al128(WB);             // NMS F planes of m
  static constexpr size_t o_s2z = o_mr + NMS * al128(FB);      // z sums of q^2 (int64)
  static constexpr size_t o_xb1 = o_s2z + 8 * (size_t)WY * WXP;   // x sums of q (int64)
  static constexpr size_t o_xb2 = o_xb1 + 8 * (size_t)WY * XBS;  // x sums of q^2 (int64)
  static constexpr size_t o_s1z = o_xb2 + 8 * (size_t)WY * XBS;  // z sums of q (int32)
  static constexpr size_t o_dr = al128(o_s1z + 4 * (size_t)WY * WXP);   // 3 F planes of d
  static constexpr size_t o_red = o_dr + 12 * (size_t)FN;      // norm partials of the warps
  static constexpr size_t o_bar = (o_red + 8 * (NT / 32) + 7) & ~(size_t)7;   // the mbarrier
  static constexpr size_t bytes = o_bar + 8;
  // W boxes the warm-up burst stages at once, over every buffer below o_red
  static constexpr int WST = (int)(o_red / al128(WB));
  static_assert(WST >= 2, "staging area");
};

// One march of tile (bx, by) over output planes [z0, z1).  pa is the phase
// parity of the copy barrier, carried over the marches of a CTA (every phase
// armed in a march is awaited in it); acc0, acc1 gather sum |dr| and sum |r|.
// Returns false when a copy wait gave up: the CTA must stop.
template <int H, int TX, int TY, int MODE = kModeIterate>
__device__ __forceinline__ bool wide_march(const BoxArgs& a, int bx, int by, int z0, int z1,
                                           const CUtensorMap* map_w, const CUtensorMap* map_f, unsigned char* smem,
                                           uint32_t& pa, float& acc0, float& acc1) {
  using B = WideLayout<H, TX, TY>;
  constexpr int NT = B::NT;
  int* err = a.err ? a.err : &g_wide_err;
  float* wn = reinterpret_cast<float*>(smem + B::o_wn);
  float* wo = reinterpret_cast<float*>(smem + B::o_wo);
  float* mring = reinterpret_cast<float*>(smem + B::o_mr);
  long long* s2z = reinterpret_cast<long long*>(smem + B::o_s2z);
  long long* xb1 = reinterpret_cast<long long*>(smem + B::o_xb1);
  long long* xb2 = reinterpret_cast<long long*>(smem + B::o_xb2);
  int* s1z = reinterpret_cast<int*>(smem + B::o_s1z);
  float* dring = reinterpret_cast<float*>(smem + B::o_dr);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + B::o_bar);

  const int tid = threadIdx.x;
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int plane = nx * ny;                  // 3 N < 2^31 is checked on the host
  const int N = plane * nz;
  const int x0 = bx * TX, y0 = by * TY;
  // the SSD adjoint and the mask modes write their outputs at the centre plane
  // itself; the iteration mode's force of plane z reads d at z - 1 .. z + 1
  constexpr bool ADJ = MODE == kModeSsdAdjoint || MODE == kModeMaskAB;
  static_assert(MODE == kModeIterate || ADJ, "wide pass modes");
  // planes whose moments are needed
  const int zc_lo = ADJ ? z0 : max(0, z0 - 1), zc_hi = ADJ ? z1 - 1 : min(nz - 1, z1);
  const int zi0 = max(0, zc_lo - H);          // first plane summed in z
  const int zw = zc_lo + H;                   // first step with a centre plane
  // the last step: the adjoint's last centre plane z1 - 1; the force of plane
  // z1 - 1 comes in the step of centre z1 (past the volume at its end)
  const int zi1 = ADJ ? z1 - 1 + H : z1 + H;
  const float qs = a.qscale, inv_qs = a.inv_qscale, vfl = a.var_floor;
  const bool dbl = a.force_mode == DISC_FORCE_DOUBLE;
  const float keep = a.u_is_dr ? 0.0f : 1.0f;   // u = keep r + dr

  auto bytes_a = [&](int zi) -> uint32_t {
    const int zc = zi - H;
    return (zi < nz ? B::WB : 0u) + (zi - (2 * H + 1) >= zi0 ? B::WB : 0u) +
           (zc >= zc_lo && zc <= zc_hi ? B::FB : 0u);
  };
  auto issue_a = [&](int zi) {                // thread 0 only
    const uint32_t nb = bytes_a(zi);
    if (nb == 0) return;
    mbar_expect_tx(bar, zi == zw ? nb + a.stall_tx : nb);
    const int zo = zi - (2 * H + 1), zc = zi - H;
    // the entering plane is read again when it is the centre plane and when it
    // leaves the window: kept in L2; the leaving plane's lines are done
    if (zi < nz) tma_load_3d_hint(wn, map_w, x0 - B::XW, y0 - 1 - H, zi, bar, l2_policy_evict_last());
    if (zo >= zi0) tma_load_3d_hint(wo, map_w, x0 - B::XW, y0 - 1 - H, zo, bar, l2_policy_evict_first());
    if (zc >= zc_lo && zc <= zc_hi)
      tma_load_3d(mring + ((unsigned)zc % B::NMS) * B::MS, map_f, x0 - B::XF, y0 - 1, zc, bar);
  };
  // a wait for phase pa that gives up stops the CTA (after its copies drain)
  auto wait_a = [&](bool armed) -> bool {
    int bad = 0;
    if (armed && tid == 0) bad = !mbar_wait(bar, pa);
    if (__syncthreads_or(bad)) {
      if (tid == 0) {
        atomicOr(err, 1);
        mbar_wait(bar, pa);                   // bounded: let this CTA's copies drain
      }
      __syncthreads();
      return false;
    }
    if (armed) pa ^= 1u;
    return true;
  };

  // ---- per-thread maps, fixed for the march -----------------------------------
  // W column k of this thread: W box index << 16 | z-sum index (-1: none).  The
  // running z sums live in the z-sum planes themselves (registers only during
  // the warm-up), which keeps the march's register state small.
  int cmap[B::K1];
  static_assert(B::WXT * B::WY < 65536 && B::WXP * B::WY < 65536, "packed column map");
#pragma unroll
  for (int k = 0; k < B::K1; ++k) {
    const int e = tid + k * NT;
    const int wy = e / B::WX, wx = e - wy * B::WX;
    cmap[k] = e < B::WN ? ((wy * B::WXT + wx + B::WOFF) << 16) | (wy * B::WXP + wx) : -1;
  }
  // y task of this thread: F column fx, rows fy0 .. fy0 + SY - 1
  const int ty_task = tid < B::NSY * B::FX ? tid : -1;
  const int sy_ = tid / B::FX, fx_y = tid - sy_ * B::FX;
  const int fy0 = sy_ * B::SY;
  const int gx_y = x0 - 1 + fx_y;
  const bool ycol = ty_task >= 0 && gx_y >= 0 && gx_y < nx;
  const bool xin_y = gx_y >= H && gx_y < nx - H;
  const int nxc_y = box_count(gx_y, nx, H);
  // force stage: the x quad gxq .. gxq + 3 of tile row oyq (nx is a multiple of 4:
  // a quad lies wholly inside or outside the volume, and holds no face of the
  // volume but at its first or last voxel, as nx >= 8)
  const int oxq = 4 * (tid % B::QX), oyq = tid / B::QX;
  const int gxq = x0 + oxq, gyq = y0 + oyq;
  const bool qin = gxq < nx && gyq < ny;
  const int fq = (oyq + 1) * B::FXT + oxq + 1 + B::FO;   // F index of the quad's first voxel (16-byte aligned)
  const bool xlo = gxq > 0, xhi = gxq + 3 < nx - 1;      // neighbours beyond the quad's ends exist
  const float sx0 = xlo ? 0.5f : 1.0f, sx3 = xhi ? 0.5f : 1.0f;
  const int yl = gyq > 0 ? -B::FXT : 0, yh = gyq < ny - 1 ? B::FXT : 0;
  const float syq = diff_scale(gyq, ny);

  // ---- warm-up: planes zi0 .. zw - 1 only enter the z sums; they arrive as
  // bursts of W boxes over the buffers the march has not used yet, one copy wait
  // per burst, and are summed in the order the march would have summed them
  {
    int s1r[B::K1];
    long long s2r[B::K1];
#pragma unroll
    for (int k = 0; k < B::K1; ++k) {
      s1r[k] = 0;
      s2r[k] = 0;
    }
    fence_proxy_async();                      // earlier generic writes of the staging area
    __syncthreads();
    const int zb_end = min(zw, nz);
    for (int zb = zi0; zb < zb_end; zb += B::WST) {
      const int nb = min(B::WST, zb_end - zb);
      if (tid == 0) {
        mbar_expect_tx(bar, (uint32_t)nb * B::WB);
        for (int j = 0; j < nb; ++j)
          tma_load_3d(smem + j * al128(B::WB), map_w, x0 - B::XW, y0 - 1 - H, zb + j, bar);
      }
      if (!wait_a(true)) return false;
      for (int j = 0; j < nb; ++j) {
        const float* wj = reinterpret_cast<const float*>(smem + j * al128(B::WB));
#pragma unroll
        for (int k = 0; k < B::K1; ++k) {
          if (cmap[k] < 0) continue;
          const int qn = __float2int_rn(wj[cmap[k] >> 16] * qs);
          s1r[k] += qn;
          s2r[k] += (long long)qn * qn;
        }
      }
      __syncthreads();                        // the staging area is consumed
    }
    // the z-sum planes (inside the staging area) take over the running sums
#pragma unroll
    for (int k = 0; k < B::K1; ++k) {
      if (cmap[k] < 0) continue;
      s1z[cmap[k] & 0xffff] = s1r[k];
      s2z[cmap[k] & 0xffff] = s2r[k];
    }
  }
  if (tid == 0) issue_a(zw);

  int zc3 = ((zw - H) % 3 + 3) % 3;           // ring slot of the centre plane's d
  for (int zi = zw; zi <= zi1; ++zi, zc3 = (zc3 == 2 ? 0 : zc3 + 1)) {
    const int zc = zi - H;                    // centre plane of the patch window
    const bool do2 = zc >= zc_lo && zc <= zc_hi;
    const int zf = zc - 1;                    // plane whose force is computed this step
    const bool do3 = !ADJ && zf >= z0 && zf < z1;
    // ---- loads into registers for this step: zs of the y task, r of the force --
    float zsr[B::SY];
    if (do2 && ycol) {
      const float* zp = a.zs + (size_t)zc * plane + gx_y;
#pragma unroll
      for (int j = 0; j < B::SY; ++j) {
        const int gy = y0 - 1 + fy0 + j;
        zsr[j] = (fy0 + j < B::FY && gy >= 0 && gy < ny)
                     ? ldcs_in(a.zs, (long long)(zp - a.zs) + (long long)gy * nx, N)
                     : 0.0f;
      }
    }
    float4 rq[3];                              // r of the force quad, components x, y, z
    if (do3 && qin) {
      const long long q0 = ((long long)zf * plane + (long long)gyq * nx + gxq) / 4;
      const float4* r4 = reinterpret_cast<const float4*>(a.r);
#pragma unroll
      for (int c = 0; c < 3; ++c) rq[c] = ldcs_in(r4, q0 + (long long)c * (N / 4), 3LL * (N / 4));
    }
    // ---- the step's copies have landed --------------------------------------
    if (!wait_a(bytes_a(zi) != 0)) return false;

    // ---- stage 1: z sliding sums of the W columns -----------------------------
    const bool has_new = zi < nz, has_old = zi - (2 * H + 1) >= zi0;
#pragma unroll
    for (int k = 0; k < B::K1; ++k) {
      if (cmap[k] < 0) continue;
      const int bi = cmap[k] >> 16, si = cmap[k] & 0xffff;
      const float vn = has_new ? wn[bi] : 0.0f;
      const float vo = has_old ? wo[bi] : 0.0f;
      const int qn = __float2int_rn(vn * qs), qo = __float2int_rn(vo * qs);
      s1z[si] += qn - qo;
      s2z[si] += (long long)(qn - qo) * (long long)(qn + qo);   // q_n^2 - q_o^2
    }
    __syncthreads();
    if (tid == 0 && zi < zi1) issue_a(zi + 1);   // the W boxes are consumed
    if (!do2 && !do3) continue;                 // uniform

    if (do2) {
      // ---- stage 2a: x window sums, sliding, one task per (segment, W row) -----
      if (tid < B::NSX * B::WY) {
        const int sg = tid / B::WY, wy = tid - sg * B::WY;
        const int fx0 = sg * B::SX;
        const int* r1 = s1z + wy * B::WXP + fx0;
        const long long* r2 = s2z + wy * B::WXP + fx0;
        long long b1 = tree_sum<2 * H + 1, int>(r1, 1), b2 = tree_sum<2 * H + 1, long long>(r2, 1);
        long long* o1 = xb1 + wy * B::XBS + fx0;
        long long* o2 = xb2 + wy * B::XBS + fx0;
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

      // ---- stage 2b: y window sums, sliding; moments and correction ------------
      if (ycol) {
        const bool zin = zc >= H && zc < nz - H;
        const int nzc = box_count(zc, nz, H);
        const bool out_plane = zc >= z0 && zc < z1;
        const float* mr = mring + ((unsigned)zc % B::NMS) * B::MS;
        float* dcur = dring + zc3 * B::FN;
        long long b1 = tree_sum<2 * H + 1, long long>(xb1 + fy0 * B::XBS + fx_y, B::XBS);
        long long b2 = tree_sum<2 * H + 1, long long>(xb2 + fy0 * B::XBS + fx_y, B::XBS);
#pragma unroll
        for (int j = 0; j < B::SY; ++j) {
          const int fy = fy0 + j;
          if (fy >= B::FY) break;
          if (j > 0) {
            b1 += xb1[(fy + 2 * H) * B::XBS + fx_y] - xb1[(fy - 1) * B::XBS + fx_y];
            b2 += xb2[(fy + 2 * H) * B::XBS + fx_y] - xb2[(fy - 1) * B::XBS + fx_y];
          }
          const int gy = y0 - 1 + fy;
          if (gy < 0 || gy >= ny) continue;
          int n;
          float inv_n;
          if (xin_y && zin && gy >= H && gy < ny - H) {
            n = B::NP;
            inv_n = 1.0f / (float)B::NP;
          } else {
            n = nxc_y * box_count(gy, ny, H) * nzc;
            inv_n = 1.0f / (float)n;
          }
          const int fi = fy * B::FXT + fx_y + B::FO;
          const float vc = mr[fi];
          float dc, sg_;
          patch_moments(b1, b2, n, inv_n, __float2int_rn(vc * qs), inv_qs, vfl, dc, sg_);
          const float d = fmaf(zsr[j], sg_, dc);   // I'_s - I_m^(k)
          if constexpr (MODE == kModeMaskAB) {
            // a, b, xi of Eqs. 5-7 at the tile's own voxels (or the ratio alone)
            if (out_plane && fx_y >= 1 && fx_y <= TX && fy >= 1 && fy <= TY)
              mask_epilogue(a, (size_t)zc * plane + (size_t)gy * nx + gx_y, vc, dc, sg_, zsr[j]);
          } else if constexpr (MODE == kModeSsdAdjoint) {
            // the SSD loss and the adjoint coefficients at the tile's own voxels
            if (out_plane && fx_y >= 1 && fx_y <= TX && fy >= 1 && fy <= TY) {
              acc0 = fmaf(d, d, acc0);
              const float D = -2.0f * d;
              const float A = -D * inv_n;
              const float Bc = sg_ > 0.0f ? -D * zsr[j] * inv_n / sg_ : 0.0f;
              const long long gz = (long long)zc * plane + (long long)gy * nx + gx_y;
              st_in(a.out, gz, 4LL * N, A);
              st_in(a.out, (long long)N + gz, 4LL * N, Bc);
              st_in(a.out, 2LL * N + gz, 4LL * N, Bc * (vc + dc));
              st_in(a.out, 3LL * N + gz, 4LL * N, D);
            }
          } else {
            dcur[fi] = d;
            if (a.f_tap && out_plane && fx_y >= 1 && fx_y <= TX && fy >= 1 && fy <= TY)
              st_in(a.f_tap, (long long)zc * plane + (long long)gy * nx + gx_y, N, d);
          }
        }
      }
    }
    if (do3) {
      __syncthreads();
      // ---- stage 3: demons force (Eq. 1) and update of plane zf = zc - 1 ---------
      const bool zlo = zf > 0, zhi = zf < nz - 1;
      const float sz = diff_scale(zf, nz);
      const int s_m1 = zc3 == 2 ? 0 : zc3 + 1;      // slot of zc - 2
      const int s_0 = zc3 == 0 ? 2 : zc3 - 1;       // slot of zc - 1 = zf
      const float* dp = dring + s_0 * B::FN;
      const float* dzm = dring + (zlo ? s_m1 : s_0) * B::FN;
      const float* dzp = dring + (zhi ? zc3 : s_0) * B::FN;
      const float* mp = mring + ((unsigned)zf % B::NMS) * B::MS;
      const float* mzm = mring + ((unsigned)(zlo ? zf - 1 : zf) % B::NMS) * B::MS;
      const float* mzp = mring + ((unsigned)(zhi ? zf + 1 : zf) % B::NMS) * B::MS;
      const bool nin = a.norm_hi <= a.norm_lo || (zf >= a.norm_lo && zf < a.norm_hi);
      if (qin) {
        // the quad's values and its neighbours': 16-byte loads of whole quads
        const float4 dc = *reinterpret_cast<const float4*>(dp + fq);
        const float4 mc = *reinterpret_cast<const float4*>(mp + fq);
        const float dl = dp[fq + (xlo ? -1 : 0)], dr4 = dp[fq + (xhi ? 4 : 3)];
        const float ml = mp[fq + (xlo ? -1 : 0)], mr4 = mp[fq + (xhi ? 4 : 3)];
        const float4 dym = *reinterpret_cast<const float4*>(dp + fq + yl);
        const float4 dyp = *reinterpret_cast<const float4*>(dp + fq + yh);
        const float4 mym = *reinterpret_cast<const float4*>(mp + fq + yl);
        const float4 myp = *reinterpret_cast<const float4*>(mp + fq + yh);
        const float4 dz0 = *reinterpret_cast<const float4*>(dzm + fq);
        const float4 dz1 = *reinterpret_cast<const float4*>(dzp + fq);
        const float4 mz0 = *reinterpret_cast<const float4*>(mzm + fq);
        const float4 mz1 = *reinterpret_cast<const float4*>(mzp + fq);
        const float dcv[4] = {dc.x, dc.y, dc.z, dc.w}, mcv[4] = {mc.x, mc.y, mc.z, mc.w};
        const float dymv[4] = {dym.x, dym.y, dym.z, dym.w}, dypv[4] = {dyp.x, dyp.y, dyp.z, dyp.w};
        const float mymv[4] = {mym.x, mym.y, mym.z, mym.w}, mypv[4] = {myp.x, myp.y, myp.z, myp.w};
        const float dz0v[4] = {dz0.x, dz0.y, dz0.z, dz0.w}, dz1v[4] = {dz1.x, dz1.y, dz1.z, dz1.w};
        const float mz0v[4] = {mz0.x, mz0.y, mz0.z, mz0.w}, mz1v[4] = {mz1.x, mz1.y, mz1.z, mz1.w};
        const float rxv[4] = {rq[0].x, rq[0].y, rq[0].z, rq[0].w};
        const float ryv[4] = {rq[1].x, rq[1].y, rq[1].z, rq[1].w};
        const float rzv[4] = {rq[2].x, rq[2].y, rq[2].z, rq[2].w};
        float ux[4], uy[4], uz[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          // x neighbours: inside the quad, or beyond its ends (the voxel itself at a face)
          const float dxm = e == 0 ? dl : dcv[e - 1], dxp = e == 3 ? dr4 : dcv[e + 1];
          const float mxm = e == 0 ? ml : mcv[e - 1], mxp = e == 3 ? mr4 : mcv[e + 1];
          const float sx = e == 0 ? sx0 : (e == 3 ? sx3 : 0.5f);
          const Dr dr = demons_dr(dcv[e], sx, dxp - dxm, mxp - mxm, syq, dypv[e] - dymv[e], mypv[e] - mymv[e],
                                  sz, dz1v[e] - dz0v[e], mz1v[e] - mz0v[e], dbl);
          ux[e] = fmaf(keep, rxv[e], dr.x);
          uy[e] = fmaf(keep, ryv[e], dr.y);
          uz[e] = fmaf(keep, rzv[e], dr.z);
          acc0 += nin ? norm3(dr.x, dr.y, dr.z) : 0.0f;
          acc1 += nin ? norm3(rxv[e], ryv[e], rzv[e]) : 0.0f;
        }
        float4* o4 = reinterpret_cast<float4*>(a.out);
        const long long q0 = ((long long)zf * plane + (long long)gyq * nx + gxq) / 4, nq = 3LL * (N / 4);
        stcs_in(o4, q0, nq, make_float4(ux[0], ux[1], ux[2], ux[3]));
        stcs_in(o4, q0 + N / 4, nq, make_float4(uy[0], uy[1], uy[2], uy[3]));
        stcs_in(o4, q0 + 2LL * (N / 4), nq, make_float4(uz[0], uz[1], uz[2], uz[3]));
      }
    }
    // the next step's stage 1 rewrites the z sums and the next stage 2b a d plane
    // that stage 3 may still read: the next step's barriers separate them
  }
  return true;
}

// Per-CTA end: the CTA's partial sums of sum |dr| and sum |r| (fixed order).
__device__ __forceinline__ void write_partials(float acc0, float acc1, float* red, float* partials, size_t part) {
  for (int off = 16; off > 0; off >>= 1) {
    acc0 += __shfl_down_sync(0xffffffffu, acc0, off);
    acc1 += __shfl_down_sync(0xffffffffu, acc1, off);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    red[wid] = acc0;
    red[kWideThreads / 32 + wid] = acc1;
  }
  __syncthreads();
  if (threadIdx.x == 0 && partials != nullptr) {
    float t0 = 0.0f, t1 = 0.0f;
    for (int w = 0; w < kWideThreads / 32; ++w) {
      t0 += red[w];
      t1 += red[kWideThreads / 32 + w];
    }
    partials[2 * part] = t0;
    partials[2 * part + 1] = t1;
  }
}

template <int H, int TX, int TY>
__device__ __forceinline__ bool wide_setup(unsigned char* smem, int* err) {
  using B = WideLayout<H, TX, TY>;
  if ((smem_addr(smem) & 127u) != 0u) {
    if (threadIdx.x == 0) atomicOr(err ? err : &g_wide_err, 2);
    return false;
  }
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + B::o_bar);
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_proxy_async();
  }
  __syncthreads();
  return true;
}

// One volume: CTA c marches the planes [c P / G, (c + 1) P / G) of the
// sequence of all P = tiles x nz (tile, plane) pairs, tile after tile (at most
// a few tiles per CTA), G = gridDim.x.
template <int H, int TX, int TY, int MODE>
__global__ void __launch_bounds__(kWideThreads, 2)
    k_box_wide(const BoxArgs a, const __grid_constant__ CUtensorMap map_w, const __grid_constant__ CUtensorMap map_f,
               int tiles_x, int tiles_y) {
  using B = WideLayout<H, TX, TY>;
  extern __shared__ __align__(128) unsigned char smem[];
  pdl_wait();
  pdl_release();
  if (a.stop != nullptr && *(volatile const int*)a.stop != 0) return;
  if (!wide_setup<H, TX, TY>(smem, a.err)) return;
  uint32_t pa = 0;
  float acc0 = 0.0f, acc1 = 0.0f;
  const long long P = (long long)tiles_x * tiles_y * a.nz;
  const long long lo = P * blockIdx.x / gridDim.x, hi = P * (blockIdx.x + 1) / gridDim.x;
  for (long long gp = lo; gp < hi;) {
    const int t = (int)(gp / a.nz), z0 = (int)(gp - (long long)t * a.nz);
    const int z1 = (int)min((long long)a.nz, (long long)z0 + (hi - gp));
    __syncthreads();                          // the previous march's reads of the buffers are done
    if (!wide_march<H, TX, TY, MODE>(a, t % tiles_x, t / tiles_x, z0, z1, &map_w, &map_f, smem, pa, acc0, acc1))
      return;
    gp += z1 - z0;
  }
  write_partials(acc0, acc1, reinterpret_cast<float*>(smem + B::o_red), a.partials, blockIdx.x);
}

// Many volumes in one launch: the (tile, plane) pairs of volume p are the
// planes [off[p], off[p + 1]) of one sequence over all volumes, which the CTAs
// share evenly as in k_box_wide; a march never crosses a volume.  The tensor
// maps of volume p are maps[2p], maps[2p + 1] (W box, F box of its m) in global
// memory.  Each CTA writes its partial sums into slot blockIdx.x of every
// volume's partials (zeros for the volumes it has no planes of), so that each
// volume's norm adds gridDim.x partials.
template <int H, int TX, int TY>
__global__ void __launch_bounds__(kWideThreads, 2)
    k_box_wide_batch(const __grid_constant__ WideBatch wb, const CUtensorMap* __restrict__ maps) {
  using B = WideLayout<H, TX, TY>;
  extern __shared__ __align__(128) unsigned char smem[];
  pdl_wait();
  pdl_release();
  if (!wide_setup<H, TX, TY>(smem, nullptr)) return;
  float* red = reinterpret_cast<float*>(smem + B::o_red);
  uint32_t pa = 0;
  const long long P = wb.off[wb.count];
  const long long lo = P * blockIdx.x / gridDim.x, hi = P * (blockIdx.x + 1) / gridDim.x;
  // volumes without planes in [lo, hi): zero partials
  if (threadIdx.x == 0) {
    for (int p = 0; p < wb.count; ++p)
      if (wb.args[p].partials != nullptr && (wb.off[p + 1] <= lo || wb.off[p] >= hi)) {
        wb.args[p].partials[2 * blockIdx.x] = 0.0f;
        wb.args[p].partials[2 * blockIdx.x + 1] = 0.0f;
      }
  }
  int p = 0;
  while (p + 1 < wb.count && wb.off[p + 1] <= lo) ++p;
  for (long long gp = lo; gp < hi && p < wb.count; ++p) {
    const BoxArgs& a = wb.args[p];
    const long long pend = min(hi, wb.off[p + 1]);
    float acc0 = 0.0f, acc1 = 0.0f;
    const CUtensorMap* mw = maps + 2 * p;
    if (threadIdx.x == 0) {
      // the maps reach the tensor-map proxy through global memory
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(mw))
                   : "memory");
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(mw + 1))
                   : "memory");
    }
    const bool stopped = a.stop != nullptr && *(volatile const int*)a.stop != 0;
    while (gp < pend) {
      const long long local = gp - wb.off[p];
      const int t = (int)(local / a.nz), z0 = (int)(local - (long long)t * a.nz);
      const int z1 = (int)min((long long)a.nz, (long long)z0 + (pend - gp));
      __syncthreads();                        // the previous march's reads of the buffers are done
      if (!stopped && !wide_march<H, TX, TY>(a, t % wb.tiles_x[p], t / wb.tiles_x[p], z0, z1, mw, mw + 1, smem, pa,
                                               acc0, acc1))
        return;
      gp += z1 - z0;
    }
    write_partials(acc0, acc1, red, a.partials, blockIdx.x);
    __syncthreads();                          // red is reused by the next volume's partials
  }
}

// ---- host side ---------------------------------------------------------------
constexpr int kMaxDevices = 64;

template <int H>
struct WideHost {
  static constexpr int TX = 32, TY = 32;
  using B = WideLayout<H, TX, TY>;
  static size_t smem() { return B::bytes; }
  static int extent(int axis) { return axis == 0 ? B::WXT : B::WY; }
  static int occupancy() {
    auto k = k_box_wide<H, TX, TY, kModeIterate>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B::bytes) != cudaSuccess ||
        cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kWideThreads, B::bytes) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return n;
  }
  template <int MODE>
  static cudaError_t launch(const BoxArgs& a, const BoxPlan& p, cudaStream_t s) {
    static int set[kMaxDevices] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    auto k = k_box_wide<H, TX, TY, MODE>;
    if (!set[dev]) {
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B::bytes);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
      if (e != cudaSuccess) return e;
      set[dev] = 1;
    }
    CUtensorMap mw{}, mf{};
    if (!tma_encode_volume(&mw, a.src, 3, a.nx, a.ny, a.nz, B::WXT, B::WY, 1) ||
        !tma_encode_volume(&mf, a.src, 3, a.nx, a.ny, a.nz, B::FXT, B::FY, 1))
      return cudaErrorInvalidValue;
    BoxArgs b = a;
    // DISC_SW_TMA_STALL: the first copy group waits for 16 bytes no copy delivers
    b.stall_tx = (test_switches() & DISC_SW_TMA_STALL) ? 16u : 0u;
    const int tx = (a.nx + TX - 1) / TX, ty = (a.ny + TY - 1) / TY;
    return launch_pdl(k, p.grid, dim3(kWideThreads), B::bytes, s, b, mw, mf, tx, ty);
  }
  static bool encode(const BoxArgs& a, CUtensorMap* m) {
    m[0] = CUtensorMap{};
    m[1] = CUtensorMap{};
    return tma_encode_volume(&m[0], a.src, 3, a.nx, a.ny, a.nz, B::WXT, B::WY, 1) &&
           tma_encode_volume(&m[1], a.src, 3, a.nx, a.ny, a.nz, B::FXT, B::FY, 1);
  }
  static cudaError_t launch_batch(const WideBatch& wb, const CUtensorMap* maps, int grid, cudaStream_t s) {
    static int set[kMaxDevices] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    auto k = k_box_wide_batch<H, TX, TY>;
    if (!set[dev]) {
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B::bytes);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
      if (e != cudaSuccess) return e;
      set[dev] = 1;
    }
    return launch_pdl(k, dim3(grid), dim3(kWideThreads), B::bytes, s, wb, maps);
  }
};

template <typename R, typename F>
R wide_dispatch(int h, R fallback, F f) {
  switch (h) {
    case 1: return f(WideHost<1>{});
    case 2: return f(WideHost<2>{});
    case 3: return f(WideHost<3>{});
    case 4: return f(WideHost<4>{});
    case 5: return f(WideHost<5>{});
    case 6: return f(WideHost<6>{});
    case 7: return f(WideHost<7>{});
    default: return fallback;
  }
}

}  // namespace

bool box_wide_ok(int nx, int ny, int nz, int hx, int hy, int hz) {
  if (hx != hy || hy != hz || hx < 1 || hx > 7) return false;
  if ((test_switches() & DISC_SW_NO_TMA) != 0u || nx % 4 != 0 || nz < 1) return false;
  const int ex = wide_dispatch<int>(hx, 0, [](auto w) { return decltype(w)::extent(0); });
  const int ey = wide_dispatch<int>(hx, 0, [](auto w) { return decltype(w)::extent(1); });
  if (ex == 0 || nx < ex || ny < ey) return false;
  return tma_encode_available();
}

size_t box_wide_smem(int h) {
  return wide_dispatch<size_t>(h, (size_t)0, [](auto w) { return decltype(w)::smem(); });
}

int box_wide_occupancy(int h) {
  return wide_dispatch<int>(h, 0, [](auto w) { return decltype(w)::occupancy(); });
}

void box_wide_tile(int* tx, int* ty) {
  *tx = WideHost<1>::TX;
  *ty = WideHost<1>::TY;
}

cudaError_t box_wide_launch(int mode, const BoxArgs& a, const BoxPlan& p, cudaStream_t s) {
  if ((((uintptr_t)a.src | (uintptr_t)a.r | (uintptr_t)a.out) & 15u) != 0u) return cudaErrorInvalidValue;
  if (mode == kModeSsdAdjoint)
    return wide_dispatch<cudaError_t>(a.hx, cudaErrorInvalidValue, [&](auto w) {
      return decltype(w)::template launch<kModeSsdAdjoint>(a, p, s);
    });
  if (mode == kModeMaskAB)
    return wide_dispatch<cudaError_t>(a.hx, cudaErrorInvalidValue, [&](auto w) {
      return decltype(w)::template launch<kModeMaskAB>(a, p, s);
    });
  if (mode != kModeIterate) return cudaErrorInvalidValue;
  return wide_dispatch<cudaError_t>(a.hx, cudaErrorInvalidValue,
                                    [&](auto w) { return decltype(w)::template launch<kModeIterate>(a, p, s); });
}

bool box_wide_encode(const BoxArgs& a, void* maps) {
  return wide_dispatch<bool>(a.hx, false,
                             [&](auto w) { return decltype(w)::encode(a, static_cast<CUtensorMap*>(maps)); });
}

cudaError_t box_wide_launch_batch(const WideBatch& wb, const void* maps, int h, int grid, cudaStream_t s) {
  if (grid < 1) return cudaSuccess;
  return wide_dispatch<cudaError_t>(h, cudaErrorInvalidValue, [&](auto w) {
    return decltype(w)::launch_batch(wb, static_cast<const CUtensorMap*>(maps), grid, s);
  });
}

cudaError_t box_wide_error(cudaStream_t s, int* flag) {
  int* dev = nullptr;
  cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&dev), g_wide_err);
  if (e != cudaSuccess) return e;
  int v = 0;
  e = cudaMemcpyAsync(&v, dev, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && v != 0) e = cudaMemsetAsync(dev, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  *flag |= v;
  return e;
}

}  // namespace disc
