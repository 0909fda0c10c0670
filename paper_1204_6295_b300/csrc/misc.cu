// Small kernels of the DISC path (sm_103a): global shift, pyramid down- and
// up-sampling, largest magnitude, and the convergence norm.

#include <cmath>

#include "internal.cuh"

namespace disc {

namespace {

constexpr int kRedThreads = 256;

// Fixed-order block sum of one double per thread (deterministic).
__device__ double block_sum_d(double v, double* sh) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
  __syncthreads();
  return s;
}

__global__ void k_max_abs(const float* __restrict__ v, int64_t n, unsigned int* out) {
  float m = 0.0f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float a = fabsf(__ldg(v + i));
    m = (a > m || a != a) ? a : m;   // a NaN wins so that it is reported
  }
  for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));   // m >= 0: bits order as values
}

// Sec. 2.3: sums of I_m and I_s, per-CTA double partials (grid-stride, fixed order)
__global__ void k_pair_sums(const float* __restrict__ a, const float* __restrict__ b, int64_t n,
                            double* part) {
  __shared__ double sh[kRedThreads / 32];
  double sa = 0.0, sb = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    sa += (double)__ldg(a + i);
    sb += (double)__ldg(b + i);
  }
  sa = block_sum_d(sa, sh);
  sb = block_sum_d(sb, sh);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = sa;
    part[2 * blockIdx.x + 1] = sb;
  }
}

// dHU = mean(I_m) - mean(I_s), one block, fixed order over the partials.
__global__ void k_shift_finalize(const double* part, int nparts, int64_t n, double* delta,
                                 float* delta_out) {
  __shared__ double sh[kRedThreads / 32];
  double sa = 0.0, sb = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
    sa += part[2 * i];
    sb += part[2 * i + 1];
  }
  sa = block_sum_d(sa, sh);
  sb = block_sum_d(sb, sh);
  if (threadIdx.x == 0) {
    const double d = (sa - sb) / (double)n;
    *delta = d;
    if (delta_out) *delta_out = (float)d;
  }
}

__global__ void k_shift_apply(const float* __restrict__ in, float* out, int64_t n, const double* delta) {
  const float d = (float)*delta;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[i] + d;
}

// Pyramid: mean over each 2x2x2 cell (in-volume voxels only).
__global__ void k_down2(const float* __restrict__ in, float* __restrict__ out, int nx, int ny, int nz,
                        int cx, int cy, int cz) {
  const int64_t nc = (int64_t)cx * cy * cz;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nc;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % cx);
    const int y = (int)((i / cx) % cy);
    const int z = (int)(i / ((int64_t)cx * cy));
    float s = 0.0f;
    int cnt = 0;
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          const int X = 2 * x + dx, Y = 2 * y + dy, Z = 2 * z + dz;
          if (X < nx && Y < ny && Z < nz) {
            s += ldg_in(in, (long long)vix(X, Y, Z, nx, ny), (long long)nx * ny * nz);
            ++cnt;
          }
        }
    st_in(out, i, nc, s / (float)cnt);
  }
}

// Coarse position of fine voxel i: (i - 0.5)/2 clamped to [0, nc-1].
__device__ __forceinline__ void up_axis(int i, int nc, int& i0, int& i1, float& t) {
  float p = 0.5f * (float)i - 0.25f;
  p = fminf(fmaxf(p, 0.0f), (float)(nc - 1));
  i0 = (int)floorf(p);
  t = p - (float)i0;
  i1 = min(i0 + 1, nc - 1);
}

__global__ void k_up2(const float* __restrict__ rc, float* __restrict__ rf, int nx, int ny, int nz,
                      int cx, int cy, int cz) {
  const int64_t nf = (int64_t)nx * ny * nz;
  const int64_t ncv = (int64_t)cx * cy * cz;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nf;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx);
    const int y = (int)((i / nx) % ny);
    const int z = (int)(i / ((int64_t)nx * ny));
    int x0, x1, y0, y1, z0, z1;
    float tx, ty, tz;
    up_axis(x, cx, x0, x1, tx);
    up_axis(y, cy, y0, y1, ty);
    up_axis(z, cz, z0, z1, tz);
    for (int c = 0; c < 3; ++c) {
      auto at = [&](int a, int b, int d) {
        return ldg_in(rc, (long long)c * ncv + (long long)vix(a, b, d, cx, cy), 3LL * ncv);
      };
      const float c00 = fmaf(tx, at(x1, y0, z0) - at(x0, y0, z0), at(x0, y0, z0));
      const float c01 = fmaf(tx, at(x1, y1, z0) - at(x0, y1, z0), at(x0, y1, z0));
      const float c10 = fmaf(tx, at(x1, y0, z1) - at(x0, y0, z1), at(x0, y0, z1));
      const float c11 = fmaf(tx, at(x1, y1, z1) - at(x0, y1, z1), at(x0, y1, z1));
      const float c0 = fmaf(ty, c01 - c00, c00), c1 = fmaf(ty, c11 - c10, c10);
      st_in(rf, c * nf + i, 3 * nf, 2.0f * fmaf(tz, c1 - c0, c0));
    }
  }
}

// l^(k) = sum|dr| / sum|r| (Sec. 2.3) from per-CTA partials; history and stop flag.
__device__ __forceinline__ void norm_finalize_body(const float* partials, int nparts, const NormState& st) {
  if (*(volatile int*)st.stop != 0) {
    if (st.use_cond && threadIdx.x == 0) cudaGraphSetConditional(st.cond, 0u);   // leave the loop
    return;
  }
  __shared__ double sh[kRedThreads / 32];
  double sdr = 0.0, sr = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
    sdr += (double)partials[2 * i];
    sr += (double)partials[2 * i + 1];
  }
  sdr = block_sum_d(sdr, sh);
  sr = block_sum_d(sr, sh);
  if (threadIdx.x == 0) {
    const int k = *st.iter;
    const float l = sr > 0.0 ? (float)(sdr / sr) : INFINITY;
    if (k < st.cap) {
      st.hist[k] = l;
      if (st.sums) {
        st.sums[2 * k] = sdr;
        st.sums[2 * k + 1] = sr;
      }
    }
    *st.iter = k + 1;
    bool stop = false;
    if (st.eps > 0.0f && k >= st.window && k < st.cap) {
      const float lp = st.hist[k - st.window];
      if (isfinite(lp) && isfinite(l) && lp - l <= st.eps) {
        *st.stop = 1;
        stop = true;
      }
    }
    if (st.use_cond) {
      const int left = *st.budget - 1;
      *st.budget = left;
      cudaGraphSetConditional(st.cond, (left > 0 && !stop) ? 1u : 0u);
    }
  }
}

__global__ void k_norm_finalize(const float* partials, int nparts, NormState st) {
  pdl_wait();
  pdl_release();
  norm_finalize_body(partials, nparts, st);
}

// One block per volume of a batch.
__global__ void k_norm_finalize_batch(const __grid_constant__ NormBatch nb) {
  pdl_wait();
  pdl_release();
  const int p = blockIdx.x;
  norm_finalize_body(nb.partials[p], nb.nparts[p], nb.st[p]);
}

__global__ void k_partials_sum(const float* partials, int nparts, int comp, double* out) {
  __shared__ double sh[kRedThreads / 32];
  double s = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += (double)partials[2 * i + comp];
  s = block_sum_d(s, sh);
  if (threadIdx.x == 0) *out = s;
}

__global__ void k_set_int(int* p, int v) { *p = v; }

int grid_for(int64_t n) {
  int64_t b = (n + kRedThreads - 1) / kRedThreads;
  if (b > 4 * 148 * 8) b = 4 * 148 * 8;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

cudaError_t launch_max_abs(const float* v, int64_t n, float* out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(float), s);
  if (e != cudaSuccess) return e;
  if (n <= 0) return cudaSuccess;
  k_max_abs<<<grid_for(n), kRedThreads, 0, s>>>(v, n, reinterpret_cast<unsigned int*>(out));
  return cudaGetLastError();
}

cudaError_t launch_global_shift(const float* Im, const float* Is, float* Is_out, int64_t n,
                                double* scratch, float* delta_out, cudaStream_t s) {
  k_pair_sums<<<kShiftBlocks, kRedThreads, 0, s>>>(Im, Is, n, scratch);
  k_shift_finalize<<<1, kRedThreads, 0, s>>>(scratch, kShiftBlocks, n, scratch + 2 * kShiftBlocks,
                                             delta_out);
  k_shift_apply<<<grid_for(n), kRedThreads, 0, s>>>(Is, Is_out, n, scratch + 2 * kShiftBlocks);
  return cudaGetLastError();
}

cudaError_t launch_down2(const float* in, float* out, int nx, int ny, int nz, cudaStream_t s) {
  const int cx = (nx + 1) / 2, cy = (ny + 1) / 2, cz = (nz + 1) / 2;
  k_down2<<<grid_for((int64_t)cx * cy * cz), kRedThreads, 0, s>>>(in, out, nx, ny, nz, cx, cy, cz);
  return cudaGetLastError();
}

cudaError_t launch_up2(const float* rc, float* rf, int nx, int ny, int nz, cudaStream_t s) {
  const int cx = (nx + 1) / 2, cy = (ny + 1) / 2, cz = (nz + 1) / 2;
  k_up2<<<grid_for((int64_t)nx * ny * nz), kRedThreads, 0, s>>>(rc, rf, nx, ny, nz, cx, cy, cz);
  return cudaGetLastError();
}

void keep_pool_memory() {
  static bool done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return;
  }
  if (done[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    unsigned long long keep = ~0ull;   // hold freed blocks for the next call instead of unmapping them
    if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) == cudaSuccess) done[dev] = true;
  }
  cudaGetLastError();
}

cudaError_t launch_set_int(int* p, int v, cudaStream_t s) {
  k_set_int<<<1, 1, 0, s>>>(p, v);
  return cudaGetLastError();
}

cudaError_t launch_norm_finalize(const float* partials, int nparts, NormState st, cudaStream_t s) {
  return launch_pdl(k_norm_finalize, dim3(1), dim3(kRedThreads), 0, s, partials, nparts, st);
}

cudaError_t launch_norm_finalize_batch(const NormBatch& nb, int count, cudaStream_t s) {
  if (count < 1) return cudaSuccess;
  return launch_pdl(k_norm_finalize_batch, dim3(count), dim3(kRedThreads), 0, s, nb);
}

cudaError_t launch_partials_sum(const float* partials, int nparts, int comp, double* out,
                                cudaStream_t s) {
  k_partials_sum<<<1, kRedThreads, 0, s>>>(partials, nparts, comp, out);
  return cudaGetLastError();
}

}  // namespace disc

// Sec. 2.3 stop rule over sums gathered outside a context (disc_norm_stop_rule):
// the arithmetic of norm_finalize_body above, on the host.
extern "C" disc_status disc_norm_stop_rule(const double* sums, int32_t count, int32_t window, float eps,
                                           float* l_out, int32_t* stop) {
  if (!sums || count < 1 || window < 1 || !stop) return DISC_ERR_ARG;
  float lp = 0.0f, l = 0.0f;
  for (int32_t k = 0; k < count; ++k) {
    const double sdr = sums[2 * k], sr = sums[2 * k + 1];
    const float v = sr > 0.0 ? (float)(sdr / sr) : INFINITY;
    if (l_out) l_out[k] = v;
    if (k == count - 1 - window) lp = v;
    if (k == count - 1) l = v;
  }
  const int32_t k = count - 1;
  *stop = (eps > 0.0f && k >= window && std::isfinite(lp) && std::isfinite(l) && lp - l <= eps) ? 1 : 0;
  return DISC_OK;
}
