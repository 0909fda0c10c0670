// Differentiable form of the DISC iteration front (sm_103a): the SSD loss
// between the warped CT and the moment-matched CBCT, and its gradient with
// respect to the displacement field by hand-written adjoint kernels.
//
//   L(r) = sum_x (m(x) - I'_s(x))^2,  m = I_m(x + r(x)),
//   I'_s = zs STD(M) + E(M)  (= a I_s + b of Eqs. 5-6; zs from the CBCT, fixed)
//
// Backward, with d = I'_s - m, D = 2 (m - I'_s) = -2 d, n the patch size:
//   A = -D / n,  B = -D zs / (n STD(M))  (0 where STD(M) = 0),  C = B E(M)
//   g_m(y) = D(y) + sum_{x in box(y)} A(x) + m(y) sum B(x) - sum C(x)
//   dL/dr(y) = g_m(y) * grad I_m at y + r(y)   (analytic trilinear derivative)
// The patch statistics are recomputed in the backward pass, not stored:
// warp -> moment pass in adjoint mode (A, B, C, D) -> truncated box sums of A,
// B, C (the separable filter kernels with unit taps and no renormalisation) ->
// the final combination below.

#include "internal.cuh"
#include "warp_dev.cuh"

namespace disc {

namespace {

constexpr int kFinalThreads = 128;

__global__ void __launch_bounds__(kFinalThreads) k_ssd_final(const float* __restrict__ Im,
                                                             const float* __restrict__ r,
                                                             const float* __restrict__ m,
                                                             const float* __restrict__ D,
                                                             const float* __restrict__ S,
                                                             float* __restrict__ grad, int nx, int ny,
                                                             int nz) {
  const int x = blockIdx.x * kFinalThreads + threadIdx.x;
  const int y = blockIdx.y, z = blockIdx.z;
  if (x >= nx) return;
  const size_t N = (size_t)nx * ny * nz;
  const size_t g = ((size_t)z * ny + y) * nx + x;
  const float gm = D[g] + S[g] + m[g] * S[N + g] - S[2 * N + g];
  float gx, gy, gz;
  warp_grad_at(Im, x, y, z, __ldg(r + g), __ldg(r + N + g), __ldg(r + 2 * N + g), nx, ny, nz, gx, gy, gz);
  grad[g] = gm * gx;
  grad[N + g] = gm * gy;
  grad[2 * N + g] = gm * gz;
}

}  // namespace

cudaError_t launch_ssd_final(const float* Im, const float* r, const float* m, const float* D,
                             const float* S, float* grad, int nx, int ny, int nz, cudaStream_t s) {
  if (ny > 65535 || nz > 65535) return cudaErrorInvalidConfiguration;
  dim3 grid((nx + kFinalThreads - 1) / kFinalThreads, ny, nz);
  k_ssd_final<<<grid, kFinalThreads, 0, s>>>(Im, r, m, D, S, grad, nx, ny, nz);
  return cudaGetLastError();
}

}  // namespace disc

using namespace disc;

namespace {

disc_status ssd_check(const float* Im, const float* zs, const float* r, int nx, int ny, int nz,
                      const int32_t patch[3], float qscale, float var_floor, int* h) {
  if (!Im || !zs || !r || !patch || !(qscale > 0.0f) || !(var_floor >= 0.0f)) return DISC_ERR_ARG;
  for (int a = 0; a < 3; ++a) {
    if (patch[a] < 1 || patch[a] > 2 * DISC_MAX_HALF_PATCH + 1 || patch[a] % 2 == 0) return DISC_ERR_ARG;
    h[a] = (patch[a] - 1) / 2;
  }
  if (nx < 1 || ny < 1 || nz < 1 || ny > 65535 || nz > 65535) return DISC_ERR_SHAPE;
  return DISC_OK;
}

int device_sms() {
  int dev = 0, sms = kNumSMs;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

BoxArgs ssd_args(const float* m, const float* zs, int nx, int ny, int nz, const int* h, float qscale,
                 float var_floor) {
  BoxArgs a{};
  a.src = m;
  a.zs = zs;
  a.nx = nx;
  a.ny = ny;
  a.nz = nz;
  a.hx = h[0];
  a.hy = h[1];
  a.hz = h[2];
  a.qscale = qscale;
  a.inv_qscale = 1.0f / qscale;
  a.var_floor = var_floor;
  return a;
}

// L(r) into *loss (device double), using m (N floats) and partials from the caller.
cudaError_t ssd_loss_into(const float* Im, const float* zs, const float* r, float* m, double* loss, int nx,
                          int ny, int nz, const int* h, float qscale, float var_floor, cudaStream_t s) {
  const BoxPlan p = box_plan(kModeSsdLoss, nx, ny, nz, h[0], h[1], h[2], device_sms());
  if (p.grid.x == 0) return cudaErrorInvalidConfiguration;
  const int nparts = (int)(p.grid.x * p.grid.y * p.grid.z);
  float* parts = nullptr;
  cudaError_t e = cudaMallocAsync(&parts, sizeof(float) * 2 * nparts, s);
  if (e != cudaSuccess) return e;
  e = launch_warp(Im, r, m, nx, ny, nz, nullptr, s);
  BoxArgs a = ssd_args(m, zs, nx, ny, nz, h, qscale, var_floor);
  a.partials = parts;
  if (e == cudaSuccess) e = box_launch(kModeSsdLoss, a, p, s);
  if (e == cudaSuccess) e = launch_partials_sum(parts, nparts, 0, loss, s);
  cudaError_t e2 = cudaFreeAsync(parts, s);
  return e != cudaSuccess ? e : e2;
}

}  // namespace

extern "C" {

disc_status disc_k_ssd_loss(const float* Im, const float* zs, const float* r, double* loss_out, int32_t nx,
                            int32_t ny, int32_t nz, const int32_t patch[3], float qscale, float var_floor,
                            void* stream) {
  int h[3];
  disc_status st = ssd_check(Im, zs, r, nx, ny, nz, patch, qscale, var_floor, h);
  if (st != DISC_OK) return st;
  if (!loss_out) return DISC_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t N = (size_t)nx * ny * nz;
  keep_pool_memory();
  float* m = nullptr;
  if (cudaMallocAsync(&m, sizeof(float) * N, s) != cudaSuccess) {
    cudaGetLastError();
    return DISC_ERR_OOM;
  }
  cudaError_t e = ssd_loss_into(Im, zs, r, m, loss_out, nx, ny, nz, h, qscale, var_floor, s);
  cudaError_t e2 = cudaFreeAsync(m, s);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorInvalidConfiguration ? DISC_ERR_SHAPE : DISC_ERR_CUDA;
  }
  return DISC_OK;
}

disc_status disc_k_ssd_grad(const float* Im, const float* zs, const float* r, float* grad, double* loss_out,
                            int32_t nx, int32_t ny, int32_t nz, const int32_t patch[3], float qscale,
                            float var_floor, void* stream) {
  int h[3];
  disc_status st = ssd_check(Im, zs, r, nx, ny, nz, patch, qscale, var_floor, h);
  if (st != DISC_OK) return st;
  if (!grad || grad == r) return DISC_ERR_ARG;
  // the truncated box sums of the adjoint use the separable filter kernels, which
  // need one half size for all three axes
  if (h[0] != h[1] || h[1] != h[2] || h[0] < 1 || h[0] > 8) return DISC_ERR_SHAPE;
  const int sms = device_sms();
  GaussPlan gp = gauss_plan(nx, ny, nz, h[0], sms);
  if (gp.grid.x == 0 || !gp.queue) return DISC_ERR_SHAPE;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t N = (size_t)nx * ny * nz;
  float* work = nullptr;   // m (N) | A B C D (4N) | sums of A B C (3N) | filter scratch (3N)
  keep_pool_memory();
  if (cudaMallocAsync(&work, sizeof(float) * 11 * N, s) != cudaSuccess) {
    cudaGetLastError();
    return DISC_ERR_OOM;
  }
  float* m = work;
  float* abcd = work + N;
  float* sums = work + 5 * N;
  float* tmp = work + 8 * N;
  // the wide-tile adjoint pass on large volumes (one wave of CTAs), the 32 x 16
  // tiling otherwise
  const BoxPlan p = box_plan_wide_mode(kModeSsdAdjoint, nx, ny, nz, h[0], h[1], h[2], sms, m, abcd);
  if (p.grid.x == 0) {
    cudaFreeAsync(work, s);
    return DISC_ERR_SHAPE;
  }
  const int nparts = (int)(p.grid.x * p.grid.y * p.grid.z);
  float* parts = nullptr;   // the loss from the adjoint pass's own d (one pass for both)
  cudaError_t e = loss_out ? cudaMallocAsync(&parts, sizeof(float) * 2 * nparts, s) : cudaSuccess;
  if (e == cudaSuccess) e = launch_warp(Im, r, m, nx, ny, nz, nullptr, s);
  BoxArgs a = ssd_args(m, zs, nx, ny, nz, h, qscale, var_floor);
  a.out = abcd;
  a.partials = parts;
  if (e == cudaSuccess) e = box_launch(kModeSsdAdjoint, a, p, s);
  if (e == cudaSuccess && loss_out) e = launch_partials_sum(parts, nparts, 0, loss_out, s);
  if (parts) {
    const cudaError_t ef = cudaFreeAsync(parts, s);
    if (e == cudaSuccess) e = ef;
  }
  GaussArgs g{};
  g.u = abcd;
  g.r = sums;
  g.t = tmp;
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  g.R = h[0];
  g.box_sum = 1;
  for (int k = 0; k <= 2 * h[0]; ++k) g.w[k] = 1.0f;
  if (e == cudaSuccess) e = gauss_launch(g, gp, s);
  if (e == cudaSuccess) e = launch_ssd_final(Im, r, m, abcd + 3 * N, sums, grad, nx, ny, nz, s);
  cudaError_t e2 = cudaFreeAsync(work, s);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorInvalidConfiguration ? DISC_ERR_SHAPE : DISC_ERR_CUDA;
  }
  return DISC_OK;
}

}  // extern "C"
