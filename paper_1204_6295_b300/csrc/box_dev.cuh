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
