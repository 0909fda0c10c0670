// C ABI of libdisc.so (include/disc.h): the registration context, its level
// schedule (Algorithm A1) with CUDA-graph replay of each level's iterations,
// and the kernel-level entry points.

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "internal.cuh"
#include "context.cuh"

using namespace disc;

namespace {

disc_status fail(disc_ctx* c, cudaError_t e) {
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return DISC_ERR_OOM;    // allocation failures are not sticky
  }
  if (c && c->sticky == DISC_OK) c->sticky = DISC_ERR_CUDA;
  return DISC_ERR_CUDA;
}

#define CK(expr)                                 \
  do {                                           \
    cudaError_t e_ = (expr);                     \
    if (e_ != cudaSuccess) return fail(ctx, e_); \
  } while (0)

// After the stream has been synchronised: a bulk-copy wait of a box kernel that
// timed out makes the context fail with DISC_ERR_TIMEOUT.
disc_status check_device_error(disc_ctx* ctx) {
  int flag = 0;
  CK(cudaMemcpyAsync(&flag, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
  CK(cudaStreamSynchronize(ctx->s));
  if (flag != 0) {
    if (ctx->sticky == DISC_OK) ctx->sticky = DISC_ERR_TIMEOUT;
    return DISC_ERR_TIMEOUT;
  }
  return DISC_OK;
}

#define CK_DEV(ctx)                                   \
  do {                                                \
    disc_status s_ = check_device_error(ctx);         \
    if (s_ != DISC_OK) return s_;                     \
  } while (0)

disc_status check_params(const disc_params* p) {
  if (!p) return DISC_ERR_ARG;
  for (int a = 0; a < 3; ++a)
    if (p->patch[a] < 1 || p->patch[a] > 2 * DISC_MAX_HALF_PATCH + 1 || (p->patch[a] % 2) == 0)
      return DISC_ERR_ARG;
  if (!(p->gauss_sigma > 0.0f) || !std::isfinite(p->gauss_sigma)) return DISC_ERR_ARG;
  if (p->gauss_radius < 0 || p->gauss_radius > DISC_MAX_GAUSS_RADIUS) return DISC_ERR_ARG;
  if (p->gauss_radius == 0 && std::ceil(3.0 * p->gauss_sigma) > DISC_MAX_GAUSS_RADIUS) return DISC_ERR_ARG;
  if (p->levels < 1 || p->levels > DISC_MAX_LEVELS) return DISC_ERR_ARG;
  for (int l = 0; l < p->levels; ++l)
    if (p->iters[l] < 0) return DISC_ERR_ARG;
  if (p->force_mode != DISC_FORCE_THIRION && p->force_mode != DISC_FORCE_DOUBLE) return DISC_ERR_ARG;
  if (!(p->var_floor >= 0.0f)) return DISC_ERR_ARG;
  if (p->stop_window < 1) return DISC_ERR_ARG;
  return DISC_OK;
}

void free_levels(disc_ctx* c) {
  for (int l = 0; l < DISC_MAX_LEVELS; ++l) {
    Level& v = c->lev[l];
    if (v.graph) cudaGraphExecDestroy(v.graph);
    cudaFree(v.Im);
    cudaFree(v.Is);
    cudaFree(v.zs);
    cudaFree(v.m);
    cudaFree(v.r);
    cudaFree(v.u);
    cudaFree(v.t);
    cudaFree(v.hist);
    v = Level{};
  }
  cudaFree(c->partials);
  c->partials = nullptr;
  c->max_parts = 0;
  c->have_images = false;
}

// Make the library stream wait for work already queued on the caller's stream.
cudaError_t enter(disc_ctx* c) {
  cudaError_t e = cudaEventRecord(c->ev_in, c->user);
  if (e != cudaSuccess) return e;
  return cudaStreamWaitEvent(c->s, c->ev_in, 0);
}
// Make the caller's stream wait for the work this call queued.
cudaError_t leave(disc_ctx* c) {
  cudaError_t e = cudaEventRecord(c->ev_out, c->s);
  if (e != cudaSuccess) return e;
  return cudaStreamWaitEvent(c->user, c->ev_out, 0);
}

cudaError_t memcpy_kind(void* dst, const void* src, size_t bytes, int dst_kind, int src_kind,
                        cudaStream_t s) {
  cudaMemcpyKind k;
  if (dst_kind == DISC_MEM_DEVICE && src_kind == DISC_MEM_DEVICE) k = cudaMemcpyDeviceToDevice;
  else if (dst_kind == DISC_MEM_DEVICE) k = cudaMemcpyHostToDevice;
  else if (src_kind == DISC_MEM_DEVICE) k = cudaMemcpyDeviceToHost;
  else k = cudaMemcpyHostToHost;
  return cudaMemcpyAsync(dst, src, bytes, k, s);
}

BoxArgs box_args(const disc_ctx* c, const Level& v) {
  BoxArgs a{};
  a.err = c->d_err;
  a.nx = v.nx;
  a.ny = v.ny;
  a.nz = v.nz;
  a.hx = c->hx;
  a.hy = c->hy;
  a.hz = c->hz;
  a.var_floor = c->p.var_floor;
  a.force_mode = c->p.force_mode;
  return a;
}

// Queue `n` iterations of level l (box pass, Gaussian pass, norm) on c->s.
cudaError_t queue_iterations(disc_ctx* c, int l, int n) {
  Level& v = c->lev[l];
  BoxArgs a = box_args(c, v);
  a.src = v.m;
  a.zs = v.zs;
  a.r = v.r;
  a.out = v.u;
  a.partials = c->partials;
  a.stop = c->d_stop + l;
  a.qscale = c->qs_m;
  a.inv_qscale = 1.0f / c->qs_m;
  GaussArgs g{};
  g.u = v.u;
  g.r = v.r;
  g.t = v.t;
  g.Im = v.Im;
  g.m = v.m;                // the z pass also warps I_m for the next iteration
  g.stop = c->d_stop + l;
  g.nx = v.nx;
  g.ny = v.ny;
  g.nz = v.nz;
  g.R = c->R;
  std::memcpy(g.w, c->w, sizeof(c->w));
  NormState st{v.hist, c->d_iter + l, c->d_stop + l, v.hist_cap, c->p.stop_window, c->p.stop_eps};
  const int nparts = (int)(v.pa.grid.x * v.pa.grid.y * v.pa.grid.z);
  // m for the field the first iteration starts from; later iterations get it
  // from the fused warp of the Gaussian z pass
  cudaError_t e0 = launch_warp(v.Im, v.r, v.m, v.nx, v.ny, v.nz, c->d_stop + l, c->s);
  if (e0 != cudaSuccess) return e0;
  for (int k = 0; k < n; ++k) {
    cudaError_t e = box_launch(kModeIterate, a, v.pa, c->s);
    if (e != cudaSuccess) return e;
    e = gauss_launch(g, v.pb, c->s);
    if (e != cudaSuccess) return e;
    e = launch_norm_finalize(c->partials, nparts, st, c->s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t run_iterations(disc_ctx* c, int l, int n) {
  if (n <= 0) return cudaSuccess;
  Level& v = c->lev[l];
  if (!c->use_graphs) return queue_iterations(c, l, n);
  if (v.graph == nullptr || v.graph_iters != n) {
    if (v.graph) {
      cudaGraphExecDestroy(v.graph);
      v.graph = nullptr;
    }
    cudaGraph_t gph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    e = queue_iterations(c, l, n);
    cudaError_t e2 = cudaStreamEndCapture(c->s, &gph);
    if (e != cudaSuccess) {
      if (gph) cudaGraphDestroy(gph);
      return e;
    }
    if (e2 != cudaSuccess) return e2;
    e = cudaGraphInstantiate(&v.graph, gph, 0);
    cudaGraphDestroy(gph);
    if (e != cudaSuccess) {
      v.graph = nullptr;
      return e;
    }
    v.graph_iters = n;
  }
  return cudaGraphLaunch(v.graph, c->s);
}

cudaError_t reset_level_counters(disc_ctx* c, int l) {
  cudaError_t e = cudaMemsetAsync(c->d_iter + l, 0, sizeof(int), c->s);
  if (e != cudaSuccess) return e;
  return cudaMemsetAsync(c->d_stop + l, 0, sizeof(int), c->s);
}

}  // namespace

namespace disc {

cudaError_t ctx_reset_level_counters(disc_ctx* c, int l) { return reset_level_counters(c, l); }

BoxArgs ctx_box_args(const disc_ctx* c, int l) {
  const Level& v = c->lev[l];
  BoxArgs a = box_args(c, v);
  a.src = v.m;
  a.zs = v.zs;
  a.r = v.r;
  a.out = v.u;
  a.partials = c->partials;
  a.stop = c->d_stop + l;
  a.qscale = c->qs_m;
  a.inv_qscale = 1.0f / c->qs_m;
  a.zlen = v.pa.zlen;
  return a;
}

GaussArgs ctx_gauss_args(const disc_ctx* c, int l) {
  const Level& v = c->lev[l];
  GaussArgs g{};
  g.u = v.u;
  g.r = v.r;
  g.t = v.t;
  g.Im = v.Im;
  g.m = v.m;
  g.stop = c->d_stop + l;
  g.nx = v.nx;
  g.ny = v.ny;
  g.nz = v.nz;
  g.R = c->R;
  g.zlen = v.pb.zlen;
  std::memcpy(g.w, c->w, sizeof(c->w));
  return g;
}

NormState ctx_norm_state(const disc_ctx* c, int l) {
  const Level& v = c->lev[l];
  return NormState{v.hist, c->d_iter + l, c->d_stop + l, v.hist_cap, c->p.stop_window, c->p.stop_eps};
}

}  // namespace disc

// ============================================================================
// Public API
// ============================================================================
extern "C" {

const char* disc_status_str(disc_status s) {
  switch (s) {
    case DISC_OK: return "DISC_OK";
    case DISC_ERR_ARG: return "DISC_ERR_ARG: invalid argument";
    case DISC_ERR_SHAPE: return "DISC_ERR_SHAPE: unsupported or inconsistent sizes";
    case DISC_ERR_STATE: return "DISC_ERR_STATE: call out of order or context failed";
    case DISC_ERR_OOM: return "DISC_ERR_OOM: device allocation failed";
    case DISC_ERR_CUDA: return "DISC_ERR_CUDA: CUDA runtime error";
    case DISC_ERR_TIMEOUT: return "DISC_ERR_TIMEOUT: bounded device wait gave up";
  }
  return "unknown disc_status";
}

disc_status disc_params_default(disc_params* p) {
  if (!p) return DISC_ERR_ARG;
  std::memset(p, 0, sizeof(*p));
  p->patch[0] = p->patch[1] = p->patch[2] = 3;
  p->gauss_sigma = 1.0f;
  p->gauss_radius = 0;
  p->levels = 2;
  p->iters[0] = 50;
  p->iters[1] = 50;
  p->stop_eps = 0.0f;
  p->stop_window = 10;
  p->force_mode = DISC_FORCE_THIRION;
  p->global_shift = 1;
  p->var_floor = 1e-6f;
  return DISC_OK;
}

disc_status disc_create(const disc_params* p, int device, void* cuda_stream, disc_ctx** out) {
  if (!out) return DISC_ERR_ARG;
  *out = nullptr;
  disc_status st = check_params(p);
  if (st != DISC_OK) return st;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return DISC_ERR_ARG;
  }
  DeviceGuard guard(device);
  if (!guard.ok) return DISC_ERR_CUDA;
  disc_ctx* ctx = new (std::nothrow) disc_ctx();
  if (!ctx) return DISC_ERR_OOM;
  ctx->p = *p;
  ctx->device = device;
  ctx->hx = (p->patch[0] - 1) / 2;
  ctx->hy = (p->patch[1] - 1) / 2;
  ctx->hz = (p->patch[2] - 1) / 2;
  ctx->R = gauss_radius(p->gauss_sigma, p->gauss_radius);
  gauss_taps(p->gauss_sigma, ctx->R, ctx->w);
  const char* ng = std::getenv("DISC_NO_GRAPH");
  ctx->use_graphs = !(ng && ng[0] == '1');
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  cudaError_t e = cudaStreamCreateWithFlags(&ctx->s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming);
  ctx->user = static_cast<cudaStream_t>(cuda_stream);   // NULL: the legacy default stream
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_iter, sizeof(int) * DISC_MAX_LEVELS);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_stop, sizeof(int) * (DISC_MAX_LEVELS + 1));
  if (e == cudaSuccess) ctx->d_err = ctx->d_stop + DISC_MAX_LEVELS;
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_scratch, sizeof(double) * (2 * kShiftBlocks + 2));
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_maxabs, sizeof(float) * 2);
  if (e == cudaSuccess) e = cudaMemset(ctx->d_iter, 0, sizeof(int) * DISC_MAX_LEVELS);
  if (e == cudaSuccess) e = cudaMemset(ctx->d_stop, 0, sizeof(int) * (DISC_MAX_LEVELS + 1));
  if (e != cudaSuccess) {
    disc_destroy(ctx);
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? DISC_ERR_OOM : DISC_ERR_CUDA;
  }
  *out = ctx;
  return DISC_OK;
}

disc_status disc_destroy(disc_ctx* ctx) {
  if (!ctx) return DISC_OK;
  DeviceGuard guard(ctx->device);
  if (ctx->s) cudaStreamSynchronize(ctx->s);
  free_levels(ctx);
  cudaFree(ctx->d_iter);
  cudaFree(ctx->d_stop);
  cudaFree(ctx->d_scratch);
  cudaFree(ctx->d_maxabs);
  if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
  if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
  if (ctx->s) cudaStreamDestroy(ctx->s);
  cudaGetLastError();
  delete ctx;
  return DISC_OK;
}

disc_status disc_set_images(disc_ctx* ctx, const float* ct, const float* cbct, int32_t nx, int32_t ny,
                            int32_t nz, int mem_kind) {
  if (!ctx || !ct || !cbct) return DISC_ERR_ARG;
  if (mem_kind != DISC_MEM_HOST && mem_kind != DISC_MEM_DEVICE) return DISC_ERR_ARG;
  if (ctx->sticky != DISC_OK) return DISC_ERR_STATE;
  if (nx < 1 || ny < 1 || nz < 1) return DISC_ERR_SHAPE;
  if ((int64_t)nx * ny * nz > ((int64_t)1 << 34)) return DISC_ERR_SHAPE;
  DeviceGuard guard(ctx->device);
  if (!guard.ok) return DISC_ERR_CUDA;
  const int L = ctx->p.levels;
  // level sizes and plans
  int dims[DISC_MAX_LEVELS][3];
  dims[0][0] = nx;
  dims[0][1] = ny;
  dims[0][2] = nz;
  for (int l = 1; l < L; ++l)
    for (int a = 0; a < 3; ++a) dims[l][a] = (dims[l - 1][a] + 1) / 2;
  const bool same = ctx->have_images && ctx->nx == nx && ctx->ny == ny && ctx->nz == nz;
  if (!same) {
    free_levels(ctx);
    int max_parts = 1;
    for (int l = 0; l < L; ++l) {
      Level& v = ctx->lev[l];
      v.nx = dims[l][0];
      v.ny = dims[l][1];
      v.nz = dims[l][2];
      v.N = (size_t)v.nx * v.ny * v.nz;
      v.pa = box_plan(kModeIterate, v.nx, v.ny, v.nz, ctx->hx, ctx->hy, ctx->hz, ctx->num_sms);
      v.pb = gauss_plan(v.nx, v.ny, v.nz, ctx->R, ctx->num_sms);
      BoxPlan ps = box_plan(kModeStatic, v.nx, v.ny, v.nz, ctx->hx, ctx->hy, ctx->hz, ctx->num_sms);
      if (v.pa.grid.x == 0 || v.pb.grid.x == 0 || ps.grid.x == 0) {
        free_levels(ctx);
        return DISC_ERR_SHAPE;   // patch or radius too large for shared memory
      }
      const int np = (int)(v.pa.grid.x * v.pa.grid.y * v.pa.grid.z);
      if (np > max_parts) max_parts = np;
      v.hist_cap = ctx->p.iters[L - 1 - l] > 0 ? ctx->p.iters[L - 1 - l] : 1;
      cudaError_t e = cudaMalloc(&v.Im, v.N * sizeof(float));
      if (e == cudaSuccess) e = cudaMalloc(&v.Is, v.N * sizeof(float));
      if (e == cudaSuccess) e = cudaMalloc(&v.zs, v.N * sizeof(float));
      if (e == cudaSuccess) e = cudaMalloc(&v.m, v.N * sizeof(float));
      if (e == cudaSuccess) e = cudaMalloc(&v.r, 3 * v.N * sizeof(float));
      if (e == cudaSuccess) e = cudaMalloc(&v.u, 3 * v.N * sizeof(float));
      if (e == cudaSuccess) e = cudaMalloc(&v.t, 3 * v.N * sizeof(float));
      if (e == cudaSuccess) e = cudaMalloc(&v.hist, v.hist_cap * sizeof(float));
      if (e != cudaSuccess) {
        free_levels(ctx);
        return fail(ctx, e);
      }
    }
    cudaError_t e = cudaMalloc(&ctx->partials, sizeof(float) * 2 * max_parts);
    if (e != cudaSuccess) {
      free_levels(ctx);
      return fail(ctx, e);
    }
    ctx->max_parts = max_parts;
    ctx->nx = nx;
    ctx->ny = ny;
    ctx->nz = nz;
    ctx->L = L;
  } else {
    for (int l = 0; l < L; ++l) {
      if (ctx->lev[l].graph) cudaGraphExecDestroy(ctx->lev[l].graph);
      ctx->lev[l].graph = nullptr;
      ctx->lev[l].graph_iters = 0;
    }
  }
  ctx->have_images = true;
  CK(enter(ctx));
  Level& f = ctx->lev[0];
  CK(memcpy_kind(f.Im, ct, f.N * sizeof(float), DISC_MEM_DEVICE, mem_kind, ctx->s));
  CK(memcpy_kind(f.Is, cbct, f.N * sizeof(float), DISC_MEM_DEVICE, mem_kind, ctx->s));
  if (ctx->p.global_shift)
    CK(launch_global_shift(f.Im, f.Is, f.Is, (int64_t)f.N, ctx->d_scratch, nullptr, ctx->s));
  for (int l = 1; l < L; ++l) {
    const Level& a = ctx->lev[l - 1];
    CK(launch_down2(a.Im, ctx->lev[l].Im, a.nx, a.ny, a.nz, ctx->s));
    CK(launch_down2(a.Is, ctx->lev[l].Is, a.nx, a.ny, a.nz, ctx->s));
  }
  // fixed-point scales from the largest magnitudes at the finest level
  CK(launch_max_abs(f.Im, (int64_t)f.N, ctx->d_maxabs, ctx->s));
  CK(launch_max_abs(f.Is, (int64_t)f.N, ctx->d_maxabs + 1, ctx->s));
  float mx[2] = {0.0f, 0.0f};
  CK(cudaMemcpyAsync(mx, ctx->d_maxabs, sizeof(mx), cudaMemcpyDeviceToHost, ctx->s));
  CK(cudaStreamSynchronize(ctx->s));
  if (!std::isfinite(mx[0]) || !std::isfinite(mx[1])) return DISC_ERR_ARG;   // NaN/Inf input
  const int32_t patch[3] = {ctx->p.patch[0], ctx->p.patch[1], ctx->p.patch[2]};
  ctx->qs_m = disc_qscale(mx[0], patch);
  ctx->qs_s = disc_qscale(mx[1], patch);
  if (ctx->qs_m == 0.0f || ctx->qs_s == 0.0f) return DISC_ERR_ARG;
  for (int l = 0; l < L; ++l) {
    Level& v = ctx->lev[l];
    BoxArgs a = box_args(ctx, v);
    a.src = v.Is;
    a.out = v.zs;
    a.qscale = ctx->qs_s;
    a.inv_qscale = 1.0f / ctx->qs_s;
    BoxPlan ps = box_plan(kModeStatic, v.nx, v.ny, v.nz, ctx->hx, ctx->hy, ctx->hz, ctx->num_sms);
    CK(box_launch(kModeStatic, a, ps, ctx->s));
  }
  const Level& c = ctx->lev[L - 1];
  CK(cudaMemsetAsync(c.r, 0, 3 * c.N * sizeof(float), ctx->s));
  for (int l = 0; l < L; ++l) CK(reset_level_counters(ctx, l));
  ctx->cur_level = L - 1;
  ctx->cur_iter = 0;
  CK(leave(ctx));
  return DISC_OK;
}

disc_status disc_iterate(disc_ctx* ctx, int32_t max_iters, int32_t* iters_done, float* last_l) {
  if (!ctx) return DISC_ERR_ARG;
  if (ctx->sticky != DISC_OK) return DISC_ERR_STATE;
  if (!ctx->have_images) return DISC_ERR_STATE;
  DeviceGuard guard(ctx->device);
  if (!guard.ok) return DISC_ERR_CUDA;
  CK(enter(ctx));
  const int L = ctx->L;
  const int l_start = ctx->cur_level;
  long long budget = max_iters < 0 ? (1LL << 40) : max_iters;
  int touched[DISC_MAX_LEVELS];
  int ntouched = 0;
  int before[DISC_MAX_LEVELS] = {0};
  bool need_counts = iters_done != nullptr || last_l != nullptr;
  if (need_counts) {
    CK(cudaMemcpyAsync(before, ctx->d_iter, sizeof(int) * DISC_MAX_LEVELS, cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
  }
  while (true) {
    const int l = ctx->cur_level;
    const int total = ctx->p.iters[L - 1 - l];
    const int left = total - ctx->cur_iter;
    if (left > 0 && budget > 0) {
      const int n = (int)(left < budget ? left : budget);
      CK(run_iterations(ctx, l, n));
      if (ntouched == 0 || touched[ntouched - 1] != l) touched[ntouched++] = l;
      ctx->cur_iter += n;
      budget -= n;
    }
    if (ctx->cur_iter >= total && l > 0) {
      // level finished: up-sample the field to the next finer level (Algorithm A1)
      const Level& fine = ctx->lev[l - 1];
      CK(launch_up2(ctx->lev[l].r, fine.r, fine.nx, fine.ny, fine.nz, ctx->s));
      CK(reset_level_counters(ctx, l - 1));
      ctx->cur_level = l - 1;
      ctx->cur_iter = 0;
      continue;
    }
    break;
  }
  if (need_counts) {
    int after[DISC_MAX_LEVELS] = {0};
    CK(cudaMemcpyAsync(after, ctx->d_iter, sizeof(int) * DISC_MAX_LEVELS, cudaMemcpyDeviceToHost, ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    CK_DEV(ctx);
    int done = 0;
    float l_last = INFINITY;
    for (int i = 0; i < ntouched; ++i) {
      const int l = touched[i];
      // a level entered during this call had its counter reset to 0
      const int b = (l == l_start) ? before[l] : 0;
      done += after[l] - b;
      if (after[l] > 0) {
        float v = INFINITY;
        const Level& lv = ctx->lev[l];
        const int k = after[l] - 1 < lv.hist_cap ? after[l] - 1 : lv.hist_cap - 1;
        CK(cudaMemcpy(&v, lv.hist + k, sizeof(float), cudaMemcpyDeviceToHost));
        l_last = v;
      }
    }
    if (iters_done) *iters_done = done;
    if (last_l) *last_l = l_last;
  }
  CK(leave(ctx));
  return DISC_OK;
}

disc_status disc_get_field(disc_ctx* ctx, float* out, int mem_kind) {
  if (!ctx || !out) return DISC_ERR_ARG;
  if (mem_kind != DISC_MEM_HOST && mem_kind != DISC_MEM_DEVICE) return DISC_ERR_ARG;
  if (ctx->sticky != DISC_OK) return DISC_ERR_STATE;
  if (!ctx->have_images) return DISC_ERR_STATE;
  DeviceGuard guard(ctx->device);
  CK(enter(ctx));
  const float* src = ctx->lev[ctx->cur_level].r;
  for (int l = ctx->cur_level; l > 0; --l) {
    const Level& fine = ctx->lev[l - 1];
    CK(launch_up2(src, fine.u, fine.nx, fine.ny, fine.nz, ctx->s));
    src = fine.u;
  }
  CK(memcpy_kind(out, src, 3 * ctx->lev[0].N * sizeof(float), mem_kind, DISC_MEM_DEVICE, ctx->s));
  if (mem_kind == DISC_MEM_HOST) CK_DEV(ctx);
  CK(leave(ctx));
  return DISC_OK;
}

disc_status disc_get_corrected(disc_ctx* ctx, float* out, int mem_kind) {
  if (!ctx || !out) return DISC_ERR_ARG;
  if (mem_kind != DISC_MEM_HOST && mem_kind != DISC_MEM_DEVICE) return DISC_ERR_ARG;
  if (ctx->sticky != DISC_OK) return DISC_ERR_STATE;
  if (!ctx->have_images) return DISC_ERR_STATE;
  DeviceGuard guard(ctx->device);
  CK(enter(ctx));
  Level& v = ctx->lev[ctx->cur_level];
  CK(launch_warp(v.Im, v.r, v.m, v.nx, v.ny, v.nz, nullptr, ctx->s));
  BoxArgs a = box_args(ctx, v);
  a.src = v.m;
  a.zs = v.zs;
  a.r = v.r;
  a.out = v.u;
  a.qscale = ctx->qs_m;
  a.inv_qscale = 1.0f / ctx->qs_m;
  BoxPlan pc = box_plan(kModeCorrected, v.nx, v.ny, v.nz, ctx->hx, ctx->hy, ctx->hz, ctx->num_sms);
  CK(box_launch(kModeCorrected, a, pc, ctx->s));
  CK(memcpy_kind(out, v.u, v.N * sizeof(float), mem_kind, DISC_MEM_DEVICE, ctx->s));
  if (mem_kind == DISC_MEM_HOST) CK_DEV(ctx);
  CK(leave(ctx));
  return DISC_OK;
}

disc_status disc_set_field(disc_ctx* ctx, int32_t level, const float* r, int mem_kind) {
  if (!ctx || !r) return DISC_ERR_ARG;
  if (mem_kind != DISC_MEM_HOST && mem_kind != DISC_MEM_DEVICE) return DISC_ERR_ARG;
  if (ctx->sticky != DISC_OK) return DISC_ERR_STATE;
  if (!ctx->have_images) return DISC_ERR_STATE;
  if (level < 0 || level >= ctx->L) return DISC_ERR_ARG;
  DeviceGuard guard(ctx->device);
  CK(enter(ctx));
  Level& v = ctx->lev[level];
  CK(memcpy_kind(v.r, r, 3 * v.N * sizeof(float), DISC_MEM_DEVICE, mem_kind, ctx->s));
  CK(reset_level_counters(ctx, level));
  ctx->cur_level = level;
  ctx->cur_iter = 0;
  if (mem_kind == DISC_MEM_HOST) CK(cudaStreamSynchronize(ctx->s));
  CK(leave(ctx));
  return DISC_OK;
}

disc_status disc_get_progress(disc_ctx* ctx, int32_t* level, int32_t* iter, int32_t dims[3]) {
  if (!ctx) return DISC_ERR_ARG;
  if (!ctx->have_images) return DISC_ERR_STATE;
  if (level) *level = ctx->cur_level;
  if (iter) *iter = ctx->cur_iter;
  if (dims) {
    const Level& v = ctx->lev[ctx->cur_level];
    dims[0] = v.nx;
    dims[1] = v.ny;
    dims[2] = v.nz;
  }
  return DISC_OK;
}

disc_status disc_get_norm_history(disc_ctx* ctx, int32_t level, float* out, int32_t cap, int32_t* count) {
  if (!ctx || !out || !count || cap < 0) return DISC_ERR_ARG;
  if (ctx->sticky != DISC_OK) return DISC_ERR_STATE;
  if (!ctx->have_images) return DISC_ERR_STATE;
  if (level < 0 || level >= ctx->L) return DISC_ERR_ARG;
  DeviceGuard guard(ctx->device);
  int k = 0;
  CK(cudaMemcpyAsync(&k, ctx->d_iter + level, sizeof(int), cudaMemcpyDeviceToHost, ctx->s));
  CK(cudaStreamSynchronize(ctx->s));
  const Level& v = ctx->lev[level];
  int n = k < v.hist_cap ? k : v.hist_cap;
  if (n > cap) n = cap;
  if (n > 0) CK(cudaMemcpy(out, v.hist, n * sizeof(float), cudaMemcpyDeviceToHost));
  *count = n;
  return DISC_OK;
}

// ============================================================================
// Kernel-level entry points
// ============================================================================

disc_status disc_k_check_error(void* stream) {
  int flag = 0;
  if (box_tma_error((cudaStream_t)stream, &flag) != cudaSuccess) {
    cudaGetLastError();
    return DISC_ERR_CUDA;
  }
  return flag != 0 ? DISC_ERR_TIMEOUT : DISC_OK;
}

float disc_qscale(float max_abs, const int32_t patch[3]) {
  if (!patch || !(max_abs >= 0.0f) || !std::isfinite(max_abs)) return 0.0f;
  double n = 1.0;
  for (int a = 0; a < 3; ++a) {
    if (patch[a] < 1) return 0.0f;
    n *= patch[a];
  }
  // |q| <= qmax keeps every patch sum of q^2 below 2^62 and z sums of q below 2^31
  double qmax = std::sqrt(std::ldexp(1.0, 62) / n);
  const double zcap = std::ldexp(1.0, 31) / (double)(patch[2] + 1);
  if (zcap < qmax) qmax = zcap;
  const double m = max_abs > 0.0f ? (double)max_abs + 1.0 : 1.0;
  int e = (int)std::floor(std::log2(qmax / m));
  if (e > 40) e = 40;
  if (e < -40) e = -40;
  return (float)std::ldexp(1.0, e);
}

disc_status disc_k_max_abs(const float* v, int64_t n, float* out, void* stream) {
  if (!v || !out || n < 0) return DISC_ERR_ARG;
  disc_ctx* ctx = nullptr;
  CK(launch_max_abs(v, n, out, (cudaStream_t)stream));
  return DISC_OK;
}

disc_status disc_k_global_shift(const float* Im, const float* Is, float* Is_out, int64_t n,
                                float* delta_out, void* stream) {
  if (!Im || !Is || !Is_out || n <= 0) return DISC_ERR_ARG;
  disc_ctx* ctx = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  double* scratch = nullptr;
  CK(cudaMallocAsync(&scratch, sizeof(double) * (2 * kShiftBlocks + 2), s));
  cudaError_t e = launch_global_shift(Im, Is, Is_out, n, scratch, delta_out, s);
  cudaError_t e2 = cudaFreeAsync(scratch, s);
  CK(e);
  CK(e2);
  return DISC_OK;
}

disc_status disc_k_downsample2(const float* in, float* out, int32_t nx, int32_t ny, int32_t nz,
                               void* stream) {
  if (!in || !out) return DISC_ERR_ARG;
  if (nx < 1 || ny < 1 || nz < 1) return DISC_ERR_SHAPE;
  disc_ctx* ctx = nullptr;
  CK(launch_down2(in, out, nx, ny, nz, (cudaStream_t)stream));
  return DISC_OK;
}

disc_status disc_k_upsample_field2(const float* rc, float* rf, int32_t nx, int32_t ny, int32_t nz,
                                   void* stream) {
  if (!rc || !rf) return DISC_ERR_ARG;
  if (nx < 1 || ny < 1 || nz < 1) return DISC_ERR_SHAPE;
  disc_ctx* ctx = nullptr;
  CK(launch_up2(rc, rf, nx, ny, nz, (cudaStream_t)stream));
  return DISC_OK;
}

static disc_status check_patch(const int32_t patch[3], int* h) {
  if (!patch) return DISC_ERR_ARG;
  for (int a = 0; a < 3; ++a) {
    if (patch[a] < 1 || patch[a] > 2 * DISC_MAX_HALF_PATCH + 1 || patch[a] % 2 == 0) return DISC_ERR_ARG;
    h[a] = (patch[a] - 1) / 2;
  }
  return DISC_OK;
}

disc_status disc_k_static_norm(const float* Is, float* zs, int32_t nx, int32_t ny, int32_t nz,
                               const int32_t patch[3], float qscale, float var_floor, void* stream) {
  int h[3];
  if (!Is || !zs || !(qscale > 0.0f) || !(var_floor >= 0.0f)) return DISC_ERR_ARG;
  disc_status st = check_patch(patch, h);
  if (st != DISC_OK) return st;
  if (nx < 1 || ny < 1 || nz < 1) return DISC_ERR_SHAPE;
  int dev = 0, sms = kNumSMs;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  BoxPlan p = box_plan(kModeStatic, nx, ny, nz, h[0], h[1], h[2], sms);
  if (p.grid.x == 0) return DISC_ERR_SHAPE;
  BoxArgs a{};
  a.src = Is;
  a.out = zs;
  a.nx = nx;
  a.ny = ny;
  a.nz = nz;
  a.hx = h[0];
  a.hy = h[1];
  a.hz = h[2];
  a.qscale = qscale;
  a.inv_qscale = 1.0f / qscale;
  a.var_floor = var_floor;
  disc_ctx* ctx = nullptr;
  CK(box_launch(kModeStatic, a, p, (cudaStream_t)stream));
  return DISC_OK;
}

disc_status disc_k_warp(const float* Im, const float* r, float* m, int32_t nx, int32_t ny, int32_t nz,
                       void* stream) {
  if (!Im || !r || !m) return DISC_ERR_ARG;
  if (nx < 1 || ny < 1 || nz < 1 || ny > 65535 || nz > 65535) return DISC_ERR_SHAPE;
  disc_ctx* ctx = nullptr;
  CK(launch_warp(Im, r, m, nx, ny, nz, nullptr, (cudaStream_t)stream));
  return DISC_OK;
}

disc_status disc_k_pass_a(const float* Im, const float* zs, const float* r, float* u, float* m_out,
                          float* d_out, double* norms_out, int32_t nx, int32_t ny, int32_t nz,
                          const int32_t patch[3], float qscale, float var_floor, int32_t force_mode,
                          void* stream) {
  int h[3];
  if (!Im || !zs || !r || !u || !(qscale > 0.0f) || !(var_floor >= 0.0f)) return DISC_ERR_ARG;
  if (u == r) return DISC_ERR_ARG;
  if (force_mode != DISC_FORCE_THIRION && force_mode != DISC_FORCE_DOUBLE) return DISC_ERR_ARG;
  disc_status st = check_patch(patch, h);
  if (st != DISC_OK) return st;
  if (nx < 1 || ny < 1 || nz < 1 || ny > 65535 || nz > 65535) return DISC_ERR_SHAPE;
  int dev = 0, sms = kNumSMs;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  BoxPlan p = box_plan(kModeIterate, nx, ny, nz, h[0], h[1], h[2], sms);
  if (p.grid.x == 0) return DISC_ERR_SHAPE;
  cudaStream_t s = (cudaStream_t)stream;
  disc_ctx* ctx = nullptr;
  const int nparts = (int)(p.grid.x * p.grid.y * p.grid.z);
  const size_t N = (size_t)nx * ny * nz;
  float* parts = nullptr;
  float* m = m_out;
  CK(cudaMallocAsync(&parts, sizeof(float) * 2 * nparts, s));
  cudaError_t e = cudaSuccess;
  if (!m) e = cudaMallocAsync(&m, sizeof(float) * N, s);
  if (e == cudaSuccess) e = launch_warp(Im, r, m, nx, ny, nz, nullptr, s);
  BoxArgs a{};
  a.src = m;
  a.zs = zs;
  a.r = r;
  a.out = u;
  a.f_tap = d_out;
  a.partials = parts;
  a.nx = nx;
  a.ny = ny;
  a.nz = nz;
  a.hx = h[0];
  a.hy = h[1];
  a.hz = h[2];
  a.qscale = qscale;
  a.inv_qscale = 1.0f / qscale;
  a.var_floor = var_floor;
  a.force_mode = force_mode;
  if (e == cudaSuccess) e = box_launch(kModeIterate, a, p, s);
  if (e == cudaSuccess && norms_out) {
    e = launch_partials_sum(parts, nparts, 0, norms_out, s);
    if (e == cudaSuccess) e = launch_partials_sum(parts, nparts, 1, norms_out + 1, s);
  }
  cudaError_t e2 = cudaFreeAsync(parts, s);
  if (!m_out && m) {
    cudaError_t e3 = cudaFreeAsync(m, s);
    if (e2 == cudaSuccess) e2 = e3;
  }
  CK(e);
  CK(e2);
  return DISC_OK;
}

disc_status disc_k_force_update(const float* m, const float* zs, const float* r, float* u, float* d_out,
                                double* norms_out, int32_t nx, int32_t ny, int32_t nz, const int32_t patch[3],
                                float qscale, float var_floor, int32_t force_mode, void* stream) {
  int h[3];
  if (!m || !zs || !r || !u || !(qscale > 0.0f) || !(var_floor >= 0.0f)) return DISC_ERR_ARG;
  if (u == r) return DISC_ERR_ARG;
  if (force_mode != DISC_FORCE_THIRION && force_mode != DISC_FORCE_DOUBLE) return DISC_ERR_ARG;
  disc_status st = check_patch(patch, h);
  if (st != DISC_OK) return st;
  if (nx < 1 || ny < 1 || nz < 1) return DISC_ERR_SHAPE;
  int dev = 0, sms = kNumSMs;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  BoxPlan p = box_plan(kModeIterate, nx, ny, nz, h[0], h[1], h[2], sms);
  if (p.grid.x == 0) return DISC_ERR_SHAPE;
  cudaStream_t s = (cudaStream_t)stream;
  disc_ctx* ctx = nullptr;
  const int nparts = (int)(p.grid.x * p.grid.y * p.grid.z);
  float* parts = nullptr;
  CK(cudaMallocAsync(&parts, sizeof(float) * 2 * nparts, s));
  BoxArgs a{};
  a.src = m;
  a.zs = zs;
  a.r = r;
  a.out = u;
  a.f_tap = d_out;
  a.partials = parts;
  a.nx = nx;
  a.ny = ny;
  a.nz = nz;
  a.hx = h[0];
  a.hy = h[1];
  a.hz = h[2];
  a.qscale = qscale;
  a.inv_qscale = 1.0f / qscale;
  a.var_floor = var_floor;
  a.force_mode = force_mode;
  cudaError_t e = box_launch(kModeIterate, a, p, s);
  if (e == cudaSuccess && norms_out) {
    e = launch_partials_sum(parts, nparts, 0, norms_out, s);
    if (e == cudaSuccess) e = launch_partials_sum(parts, nparts, 1, norms_out + 1, s);
  }
  cudaError_t e2 = cudaFreeAsync(parts, s);
  CK(e);
  CK(e2);
  return DISC_OK;
}

disc_status disc_k_gauss(const float* u, float* r, int32_t nx, int32_t ny, int32_t nz, float sigma,
                         int32_t radius, void* stream) {
  if (!u || !r || u == r || !(sigma > 0.0f) || radius < 0) return DISC_ERR_ARG;
  if (nx < 1 || ny < 1 || nz < 1) return DISC_ERR_SHAPE;
  const int R = gauss_radius(sigma, radius);
  if (R > DISC_MAX_GAUSS_RADIUS) return DISC_ERR_ARG;
  int dev = 0, sms = kNumSMs;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  GaussPlan p = gauss_plan(nx, ny, nz, R, sms);
  if (p.grid.x == 0) return DISC_ERR_SHAPE;
  GaussArgs g{};
  g.u = u;
  g.r = r;
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  g.R = R;
  gauss_taps(sigma, R, g.w);
  disc_ctx* ctx = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  float* t = nullptr;
  if (p.queue) CK(cudaMallocAsync(&t, sizeof(float) * 3 * (size_t)nx * ny * nz, s));
  g.t = t;
  cudaError_t e = gauss_launch(g, p, s);
  cudaError_t e2 = t ? cudaFreeAsync(t, s) : cudaSuccess;
  CK(e);
  CK(e2);
  return DISC_OK;
}

}  // extern "C"
