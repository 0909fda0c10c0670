// Device helpers of the cubic-patch moment kernels (box_fast.cu, box_tma.cu).
#pragma once

#include <cuda_runtime.h>

#include "internal.cuh"

namespace disc {

// 64-bit integers to float through their two 32-bit halves (two exact 32-bit
// conversions and one fused multiply-add: within 2 ulp), which keeps the
// conversion off the slow 64-bit conversion path.
static __device__ __forceinline__ float s64_to_float(long long v) {
  return fmaf((float)(int)(v >> 32), 4294967296.0f, (float)(unsigned)v);
}
static __device__ __forceinline__ float u64_to_float(unsigned long long v) {
  return fmaf((float)(unsigned)(v >> 32), 4294967296.0f, (float)(unsigned)v);
}

static __device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Sum in 64 bits of N integers p[0], p[s], ..., p[(N-1) s] as a balanced tree
// (short dependency chains; integer sums are exact in any order).
template <int N, typename T>
static __device__ __forceinline__ long long tree_sum(const T* p, int s) {
  if constexpr (N == 1) {
    return (long long)p[0];
  } else {
    return tree_sum<N / 2, T>(p, s) + tree_sum<N - N / 2, T>(p + (N / 2) * s, s);
  }
}

// Patch moments from exact integer sums S1 = sum q, S2 = sum q^2 over n voxels
// (Eq. 3, Appendix A.4): dc = E(X) - v_c with qc = rint(v_c 2^e), and
// sigma = STD(X), 0 when Var(X) <= var_floor.  With k = round(S1/n) and
// e = S1 - n k (|e| a few times n):
//   E(X) = (k + e/n) / 2^e,
//   T = sum (q - k)^2 = S2 - k (S1 + e)   (exact modulo 2^64; 0 <= T < 2^62),
//   Var(X) = (T/n - (e/n)^2) / 2^(2e).
// A constant patch gives T = e = 0, so dc = 0 and sigma = 0 exactly.
static __device__ __forceinline__ void patch_moments(long long S1, long long S2, int n, float inv_n, int qc,
                                                     float inv_qs, float var_floor, float& dc,
                                                     float& sigma) {
  const int k = __float2int_rn(s64_to_float(S1) * inv_n);
  const int e = (int)(S1 - (long long)n * k);
  const float ef = (float)e * inv_n;
  dc = ((float)(k - qc) + ef) * inv_qs;
  const unsigned long long T = (unsigned long long)S2 - (unsigned long long)(long long)k *
                                                            (unsigned long long)(S1 + e);
  const float varq = fmaf(u64_to_float(T), inv_n, -ef * ef);
  const float var = varq * (inv_qs * inv_qs);
  sigma = var > var_floor ? sqrt_approx(var) : 0.0f;
}

// Demons force of Eq. (1) (reading R1: the difference taken as I'_s - I_m^(k))
// at one voxel, with grad I'_s = grad d + grad m.  Inputs: d0 = d = I'_s - m at
// the voxel and, per axis, the difference scale s (1/2 for a central
// difference, 1 for a one-sided one at a face, 0 on an axis of one voxel) with
// the differences dd, dm of d and m between the two neighbours used.  A term
// is 0 where its denominator is <= 1e-9 (reading R11); `dbl` adds the second
// term of the double force.  Every rounding is explicit, so each kernel that
// computes the force gets the same bits.
struct Dr {
  float x, y, z;
};
static __device__ __forceinline__ Dr demons_dr(float d0, float sx, float ddx, float dmx, float sy, float ddy,
                                               float dmy, float sz, float ddz, float dmz, bool dbl) {
  const float gmx = __fmul_rn(sx, dmx), gmy = __fmul_rn(sy, dmy), gmz = __fmul_rn(sz, dmz);
  const float gfx = fmaf(sx, ddx, gmx), gfy = fmaf(sy, ddy, gmy), gfz = fmaf(sz, ddz, gmz);
  const float d2 = __fmul_rn(d0, d0);
  const float den = fmaf(gfx, gfx, fmaf(gfy, gfy, fmaf(gfz, gfz, d2)));
  const float sc = den > 1e-9f ? __fdividef(d0, den) : 0.0f;
  Dr dr{__fmul_rn(sc, gfx), __fmul_rn(sc, gfy), __fmul_rn(sc, gfz)};
  if (dbl) {
    const float den2 = fmaf(gmx, gmx, fmaf(gmy, gmy, fmaf(gmz, gmz, d2)));
    const float s2 = den2 > 1e-9f ? __fdividef(d0, den2) : 0.0f;
    dr.x = fmaf(s2, gmx, dr.x);
    dr.y = fmaf(s2, gmy, dr.y);
    dr.z = fmaf(s2, gmz, dr.z);
  }
  return dr;
}

// |v| of a 3-vector for the convergence norm l^(k) (Sec. 2.3): per-CTA float
// partial sums of these are added in a fixed order.
static __device__ __forceinline__ float norm3(float x, float y, float z) {
  return sqrt_approx(fmaf(x, x, fmaf(y, y, __fmul_rn(z, z))));
}

// Difference scale of an axis position c of n voxels (reading R10): the
// neighbours used are c + lo and c + hi (lo, hi in {-step, 0} and {0, step}).
static __device__ __forceinline__ float diff_scale(int c, int n) {
  const bool l = c > 0, h = c < n - 1;
  return (l && h) ? 0.5f : ((l || h) ? 1.0f : 0.0f);
}

// kModeMaskAB epilogue at voxel g (Eqs. 5-7; readings R17, R18), shared by the
// box kernels.  vc = m at the voxel, dc = E(M) - m, sg = STD(M), zsv = zs.
//   a = STD(M) / STD(S), b = E(M) - a E(S) with E(S) = I_s - zs STD(S);
//   xi = 1 where STD(S) = 0, |m - I_s| > HU0, or a outside [a_min, a_max].
// Unmasked voxels keep d = zs STD(M) + dc (the path's deviation form); masked
// ones start from the paper's a = b = 0 (d = -m) and stamp -1, and are counted
// for the fill passes.
static __device__ __forceinline__ void mask_epilogue(const BoxArgs& a, size_t g, float vc, float dc, float sg,
                                                     float zsv) {
  const float sd = __ldg(a.sd + g);
  if (a.ratio_only) {   // for the median a_m: defined where both patches vary (reading R18)
    a.a_out[g] = (sd > 0.0f && sg > 0.0f) ? sg / sd : -1.0f;
    return;
  }
  const float is = __ldg(a.is + g);
  const float av = sd > 0.0f ? sg / sd : 0.0f;
  const bool xi = !(sd > 0.0f) || fabsf(vc - is) > a.hu0 || av < a.a_min || av > a.a_max;
  if (!xi) {
    a.isab[g] = make_float4(is, av, (vc + dc) - av * fmaf(-zsv, sd, is), 0.0f);
    a.out[g] = fmaf(zsv, sg, dc);
    a.stamp[g] = 0;
  } else {
    a.isab[g] = make_float4(is, 0.0f, 0.0f, 0.0f);
    a.out[g] = -vc;
    a.stamp[g] = -1;
    atomicAdd(a.count, 1);
  }
}

}  // namespace disc
