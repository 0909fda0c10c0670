// Evaluation metrics of Sec. 2.4.3 (sm_103a), not on the iteration path:
// normalised mutual information and the RMSE of binary Canny edge images,
// Eq. (11).  Every floating-point step that decides an integer (a histogram
// bin, a non-maximum test, a threshold) is taken in float32 with explicitly
// rounded operations (no fused multiply-add), in a fixed order, so that the
// decisions are reproducible bit for bit:
//   NMI   bin(v) = floor((v - min) * (bins / (max - min))), clamped; entropies
//         of the joint histogram in double; NMI = 2 I / (H(A) + H(B)).
//   Canny per transverse slice: separable Gaussian (x then y, taps in order,
//         renormalised over the in-slice taps), central differences (one-sided
//         at the borders), M = sqrt(gx^2 + gy^2), non-maximum suppression along
//         the gradient direction quantised to 0/45/90/135 degrees, kept where
//         M > 1e-5 max|slice| and M >= both neighbours (outside counts as 0);
//         strong M >= t_high max_slice(M), weak M >= t_low times that;
//         hysteresis keeps weak pixels 8-connected to strong ones (repeated
//         propagation passes until none changes).

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "internal.cuh"

namespace disc {

namespace {

constexpr int kMThreads = 256;
constexpr int kMaxCannyRadius = 16;

struct CannyTaps {
  float w[2 * kMaxCannyRadius + 1];
  int R;
};

// Ordered-int encoding of floats for atomic min/max (total order on non-NaN values).
__device__ __forceinline__ int f2o(float f) {
  const int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float o2f(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

__global__ void k_minmax2(const float* __restrict__ a, const float* __restrict__ b, int64_t n, int* mm) {
  int amin = INT_MAX, amax = INT_MIN, bmin = INT_MAX, bmax = INT_MIN;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int va = f2o(__ldg(a + i)), vb = f2o(__ldg(b + i));
    amin = min(amin, va);
    amax = max(amax, va);
    bmin = min(bmin, vb);
    bmax = max(bmax, vb);
  }
  for (int off = 16; off > 0; off >>= 1) {
    amin = min(amin, __shfl_down_sync(0xffffffffu, amin, off));
    amax = max(amax, __shfl_down_sync(0xffffffffu, amax, off));
    bmin = min(bmin, __shfl_down_sync(0xffffffffu, bmin, off));
    bmax = max(bmax, __shfl_down_sync(0xffffffffu, bmax, off));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&mm[0], amin);
    atomicMax(&mm[1], amax);
    atomicMin(&mm[2], bmin);
    atomicMax(&mm[3], bmax);
  }
}

__device__ __forceinline__ int nmi_bin(float v, float mn, float mx, int bins) {
  if (mx == mn) return 0;
  const float s = __fdiv_rn((float)bins, __fsub_rn(mx, mn));
  const int b = (int)floorf(__fmul_rn(__fsub_rn(v, mn), s));
  return min(max(b, 0), bins - 1);
}

__global__ void k_joint_hist(const float* __restrict__ a, const float* __restrict__ b, int64_t n, const int* mm,
                             int bins, unsigned* hist) {
  extern __shared__ unsigned sh[];
  const int nb = bins * bins;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) sh[i] = 0u;
  __syncthreads();
  const float amin = o2f(mm[0]), amax = o2f(mm[1]), bmin = o2f(mm[2]), bmax = o2f(mm[3]);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int ia = nmi_bin(__ldg(a + i), amin, amax, bins), ib = nmi_bin(__ldg(b + i), bmin, bmax, bins);
    atomicAdd(&sh[ia * bins + ib], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nb; i += blockDim.x)
    if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

__device__ double block_sum(double v, double* sh) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
  __syncthreads();
  return s;
}

__device__ __forceinline__ double plogp(double p) { return p > 0.0 ? p * log(p) : 0.0; }

__global__ void __launch_bounds__(kMThreads) k_nmi_finish(const unsigned* hist, int bins, int64_t n, double* out) {
  __shared__ double sh[kMThreads / 32];
  const double inv = 1.0 / (double)n;
  double hab = 0.0, ha = 0.0, hb = 0.0;
  for (int i = threadIdx.x; i < bins * bins; i += blockDim.x) hab -= plogp(hist[i] * inv);
  for (int i = threadIdx.x; i < bins; i += blockDim.x) {
    double ra = 0.0, rb = 0.0;
    for (int j = 0; j < bins; ++j) {
      ra += hist[i * bins + j];
      rb += hist[j * bins + i];
    }
    ha -= plogp(ra * inv);
    hb -= plogp(rb * inv);
  }
  hab = block_sum(hab, sh);
  ha = block_sum(ha, sh);
  hb = block_sum(hb, sh);
  if (threadIdx.x == 0) *out = (ha + hb == 0.0) ? 1.0 : 2.0 * (ha + hb - hab) / (ha + hb);
}

// ---- Canny --------------------------------------------------------------------
// one separable pass along x (dir 0) or y (dir 1) of every slice
__global__ void k_canny_smooth(const float* __restrict__ in, float* __restrict__ out, int nx, int ny, int nz,
                               CannyTaps t, int dir) {
  const int64_t N = (int64_t)nx * ny * nz;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < N; g += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(g % nx), y = (int)((g / nx) % ny);
    const int c = dir == 0 ? x : y, n = dir == 0 ? nx : ny;
    const int64_t stride = dir == 0 ? 1 : nx;
    float acc = 0.0f, nrm = 0.0f;
    for (int k = -t.R; k <= t.R; ++k) {
      if (c + k < 0 || c + k >= n) continue;
      acc = __fadd_rn(acc, __fmul_rn(t.w[k + t.R], __ldg(in + g + k * stride)));
      nrm = __fadd_rn(nrm, t.w[k + t.R]);
    }
    out[g] = nrm == 1.0f ? acc : __fdiv_rn(acc, nrm);
  }
}

__device__ __forceinline__ float cdiff(const float* p, int c, int n, int64_t stride) {
  if (n < 2) return 0.0f;
  if (c == 0) return __fsub_rn(p[stride], p[0]);
  if (c == n - 1) return __fsub_rn(p[0], p[-stride]);
  return __fmul_rn(0.5f, __fsub_rn(p[stride], p[-stride]));
}

// gradient magnitude and the quantised direction: 0 x, 1 y, 2 diagonal (+,+), 3 diagonal (+,-)
__global__ void k_canny_grad(const float* __restrict__ S, float* __restrict__ M, uint8_t* __restrict__ dir, int nx,
                             int ny, int nz, float t1, float t2) {
  const int64_t N = (int64_t)nx * ny * nz;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < N; g += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(g % nx), y = (int)((g / nx) % ny);
    const float gx = cdiff(S + g, x, nx, 1), gy = cdiff(S + g, y, ny, nx);
    M[g] = __fsqrt_rn(__fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy)));
    const float ax = fabsf(gx), ay = fabsf(gy);
    uint8_t d;
    if (ay <= __fmul_rn(t1, ax)) d = 0;
    else if (ay >= __fmul_rn(t2, ax)) d = 1;
    else d = __fmul_rn(gx, gy) > 0.0f ? 2 : 3;
    dir[g] = d;
  }
}

// per slice: largest |v| (absval) or largest v; one block per slice
__global__ void __launch_bounds__(kMThreads) k_slice_max(const float* __restrict__ v, int plane, int absval,
                                                         float* out) {
  const float* p = v + (int64_t)blockIdx.x * plane;
  float m = 0.0f;
  for (int i = threadIdx.x; i < plane; i += blockDim.x) {
    const float a = absval ? fabsf(__ldg(p + i)) : __ldg(p + i);
    m = fmaxf(m, a);
  }
  for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, off));
  __shared__ float sh[kMThreads / 32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float r = 0.0f;
    for (int w = 0; w < kMThreads / 32; ++w) r = fmaxf(r, sh[w]);
    out[blockIdx.x] = r;
  }
}

// non-maximum suppression and thresholds: 0 none, 1 weak, 2 strong
__global__ void k_canny_classify(const float* __restrict__ M, const uint8_t* __restrict__ dir,
                                 const float* __restrict__ pmax, const float* __restrict__ mmax, uint8_t* cls, int nx,
                                 int ny, int nz, float t_low, float t_high) {
  const int64_t N = (int64_t)nx * ny * nz;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < N; g += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(g % nx), y = (int)((g / nx) % ny), z = (int)(g / ((int64_t)nx * ny));
    const float m = M[g];
    int dx, dy;
    switch (dir[g]) {
      case 0: dx = 1; dy = 0; break;
      case 1: dx = 0; dy = 1; break;
      case 2: dx = 1; dy = 1; break;
      default: dx = -1; dy = 1; break;
    }
    auto at = [&](int xx, int yy) {
      return (xx < 0 || xx >= nx || yy < 0 || yy >= ny) ? 0.0f : M[g + (int64_t)(yy - y) * nx + (xx - x)];
    };
    const float n1 = at(x + dx, y + dy), n2 = at(x - dx, y - dy);
    const float floor_ = __fmul_rn(1e-5f, pmax[z]);
    const bool keep = m > floor_ && m >= n1 && m >= n2;
    const float hi = __fmul_rn(t_high, mmax[z]);
    const float lo = __fmul_rn(t_low, hi);
    cls[g] = !keep ? 0 : (m >= hi ? 2 : (m >= lo ? 1 : 0));
  }
}

// one hysteresis pass: weak pixels next to an edge pixel (8-connected, in-slice) become edges
__global__ void k_hysteresis(uint8_t* cls, int nx, int ny, int nz, int* changed) {
  const int64_t N = (int64_t)nx * ny * nz;
  int any = 0;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < N; g += (int64_t)gridDim.x * blockDim.x) {
    if (cls[g] != 1) continue;
    const int x = (int)(g % nx), y = (int)((g / nx) % ny);
    bool near = false;
    for (int dy = -1; dy <= 1 && !near; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int xx = x + dx, yy = y + dy;
        if ((dx | dy) == 0 || xx < 0 || xx >= nx || yy < 0 || yy >= ny) continue;
        if (((volatile uint8_t*)cls)[g + (int64_t)dy * nx + dx] == 2) {
          near = true;
          break;
        }
      }
    if (near) {
      cls[g] = 2;
      any = 1;
    }
  }
  if (__syncthreads_or(any) && threadIdx.x == 0) atomicOr(changed, 1);
}

__global__ void k_edges_out(const uint8_t* cls, uint8_t* edges, int64_t n) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    edges[g] = cls[g] == 2 ? 1 : 0;
}

__global__ void k_count_diff(const uint8_t* a, const uint8_t* b, int64_t n, unsigned long long* count) {
  unsigned long long c = 0;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    c += ((a[g] != 0) != (b[g] != 0)) ? 1ull : 0ull;
  for (int off = 16; off > 0; off >>= 1) c += __shfl_down_sync(0xffffffffu, c, off);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

__global__ void k_rmse_finish(const unsigned long long* count, int64_t n, double* out) {
  *out = sqrt((double)*count / (double)n);
}

int blocks_for(int64_t n) {
  int64_t b = (n + kMThreads - 1) / kMThreads;
  if (b > 148 * 8) b = 148 * 8;
  return b < 1 ? 1 : (int)b;
}

}  // namespace

cudaError_t metric_nmi(const float* a, const float* b, int64_t n, int bins, double* out, cudaStream_t s) {
  if (n < 1 || bins < 2 || bins > 128) return cudaErrorInvalidValue;
  void* work = nullptr;   // 4 ordered ints, then the joint histogram
  const size_t hist_bytes = sizeof(unsigned) * bins * bins;
  cudaError_t e = cudaMallocAsync(&work, 16 + hist_bytes, s);
  if (e != cudaSuccess) return e;
  int* mm = static_cast<int*>(work);
  unsigned* hist = reinterpret_cast<unsigned*>(static_cast<char*>(work) + 16);
  const int init[4] = {INT_MAX, INT_MIN, INT_MAX, INT_MIN};
  e = cudaMemcpyAsync(mm, init, sizeof(init), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(hist, 0, hist_bytes, s);
  if (e == cudaSuccess && hist_bytes > 48 * 1024)   // up to 64 KB for 128 x 128 bins
    e = cudaFuncSetAttribute(k_joint_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hist_bytes);
  if (e == cudaSuccess) {
    k_minmax2<<<blocks_for(n), kMThreads, 0, s>>>(a, b, n, mm);
    k_joint_hist<<<blocks_for(n), kMThreads, hist_bytes, s>>>(a, b, n, mm, bins, hist);
    k_nmi_finish<<<1, kMThreads, 0, s>>>(hist, bins, n, out);
    e = cudaGetLastError();
  }
  const cudaError_t e2 = cudaFreeAsync(work, s);
  return e != cudaSuccess ? e : e2;
}

cudaError_t metric_canny(const float* img, uint8_t* edges, int nx, int ny, int nz, float sigma, float t_low,
                         float t_high, cudaStream_t s) {
  if (nx < 1 || ny < 1 || nz < 1 || !(sigma > 0.0f) || std::ceil(3.0 * sigma) > kMaxCannyRadius)
    return cudaErrorInvalidValue;
  CannyTaps t{};
  t.R = (int)std::ceil(3.0 * sigma);
  {
    double w[2 * kMaxCannyRadius + 1], sum = 0.0;
    for (int k = -t.R; k <= t.R; ++k) sum += (w[k + t.R] = std::exp(-(double)k * k / (2.0 * sigma * sigma)));
    for (int k = 0; k <= 2 * t.R; ++k) t.w[k] = (float)(w[k] / sum);
  }
  const float t1 = (float)(std::sqrt(2.0) - 1.0), t2 = (float)(std::sqrt(2.0) + 1.0);
  const int64_t N = (int64_t)nx * ny * nz;
  const int plane = nx * ny;
  char* work = nullptr;   // tmp, S, M (floats), pmax, mmax (nz floats), dir, cls (bytes), flag
  const size_t fbytes = sizeof(float) * (3 * N + 2 * (int64_t)nz);
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&work), fbytes + 2 * N + 16, s);
  if (e != cudaSuccess) return e;
  float* tmp = reinterpret_cast<float*>(work);
  float* S = tmp + N;
  float* M = S + N;
  float* pmax = M + N;
  float* mmax = pmax + nz;
  uint8_t* dir = reinterpret_cast<uint8_t*>(work + fbytes);
  uint8_t* cls = dir + N;
  int* flag = reinterpret_cast<int*>(work + ((fbytes + 2 * N + 3) & ~(size_t)3));
  const int nb = blocks_for(N);
  k_canny_smooth<<<nb, kMThreads, 0, s>>>(img, tmp, nx, ny, nz, t, 0);
  k_canny_smooth<<<nb, kMThreads, 0, s>>>(tmp, S, nx, ny, nz, t, 1);
  k_canny_grad<<<nb, kMThreads, 0, s>>>(S, M, dir, nx, ny, nz, t1, t2);
  k_slice_max<<<nz, kMThreads, 0, s>>>(img, plane, 1, pmax);
  k_slice_max<<<nz, kMThreads, 0, s>>>(M, plane, 0, mmax);
  k_canny_classify<<<nb, kMThreads, 0, s>>>(M, dir, pmax, mmax, cls, nx, ny, nz, t_low, t_high);
  e = cudaGetLastError();
  // hysteresis: propagation passes until a batch of passes changes nothing (the
  // host reads the flag after every batch; the passes are bounded by N)
  const int batch = 16;
  for (int64_t done = 0; e == cudaSuccess && done < N + batch; done += batch) {
    e = cudaMemsetAsync(flag, 0, sizeof(int), s);
    for (int k = 0; k < batch && e == cudaSuccess; ++k) {
      k_hysteresis<<<nb, kMThreads, 0, s>>>(cls, nx, ny, nz, flag);
      e = cudaGetLastError();
    }
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess || h == 0) break;
  }
  if (e == cudaSuccess) {
    k_edges_out<<<nb, kMThreads, 0, s>>>(cls, edges, N);
    e = cudaGetLastError();
  }
  const cudaError_t e2 = cudaFreeAsync(work, s);
  return e != cudaSuccess ? e : e2;
}

cudaError_t metric_edge_rmse(const uint8_t* a, const uint8_t* b, int64_t n, double* out, cudaStream_t s) {
  if (n < 1) return cudaErrorInvalidValue;
  unsigned long long* count = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&count), sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess) {
    k_count_diff<<<blocks_for(n), kMThreads, 0, s>>>(a, b, n, count);
    k_rmse_finish<<<1, 1, 0, s>>>(count, n, out);
    e = cudaGetLastError();
  }
  const cudaError_t e2 = cudaFreeAsync(count, s);
  return e != cudaSuccess ? e : e2;
}

}  // namespace disc
