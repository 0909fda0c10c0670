// C ABI of libdisc.so (include/disc.h): the registration context, its level
// schedule (Algorithm A1) with CUDA-graph replay of each level's iterations,
// and the kernel-level entry points.

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

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

disc_status check_patch(const int32_t patch[3], int* h) {
  if (!patch) return DISC_ERR_ARG;
  for (int a = 0; a < 3; ++a) {
    if (patch[a] < 1 || patch[a] > 2 * DISC_MAX_HALF_PATCH + 1 || patch[a] % 2 == 0) return DISC_ERR_ARG;
    h[a] = (patch[a] - 1) / 2;
  }
  return DISC_OK;
}

// Common argument checks and launch of the kernel-level box-pass calls.
disc_status kcheck(int32_t nx, int32_t ny, int32_t nz, const int32_t patch[3], float qscale,
                          float var_floor, int* h) {
  if (!(qscale > 0.0f) || !(var_floor >= 0.0f)) return DISC_ERR_ARG;
  disc_status st = check_patch(patch, h);
  if (st != DISC_OK) return st;
  if (nx < 1 || ny < 1 || nz < 1 || (double)nx * ny * nz * 3.0 >= 2147483647.0) return DISC_ERR_SHAPE;
  return DISC_OK;
}

BoxArgs kargs(int32_t nx, int32_t ny, int32_t nz, const int* h, float qscale, float var_floor) {
  BoxArgs a{};
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

disc_status klaunch(int mode, const BoxArgs& a, cudaStream_t s) {
  int dev = 0, sms = kNumSMs;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const BoxPlan p = box_plan(mode, a.nx, a.ny, a.nz, a.hx, a.hy, a.hz, sms);
  if (p.grid.x == 0) return DISC_ERR_SHAPE;
  if (box_launch(mode, a, p, s) != cudaSuccess) {
    cudaGetLastError();
    return DISC_ERR_CUDA;
  }
  return DISC_OK;
}

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
  if (p->mask_mode != 0 && p->mask_mode != 1) return DISC_ERR_ARG;
  if (p->smooth_mode != 0 && p->smooth_mode != 1) return DISC_ERR_ARG;
  for (int i = 0; i < 2; ++i)
    if (!(p->quant_max[i] >= 0.0f) || !std::isfinite(p->quant_max[i])) return DISC_ERR_ARG;
  if (p->norm_planes[0] < 0 || p->norm_planes[1] < 0) return DISC_ERR_ARG;
  if (p->mask_mode) {
    if (!(p->hu0_factor >= 0.0f) || !(p->a_lo >= 0.0f) || !(p->a_hi >= p->a_lo) || !(p->fill_h > 0.0f) ||
        !std::isfinite(p->hu0_factor) || !std::isfinite(p->a_hi) || !std::isfinite(p->fill_h))
      return DISC_ERR_ARG;
    for (int a = 0; a < 3; ++a)
      if (p->fill_t[a] < 1 || p->fill_t[a] > 15 || p->fill_t[a] % 2 == 0) return DISC_ERR_ARG;
    if (p->fill_passes < 1 || p->fill_passes > 1024) return DISC_ERR_ARG;
  }
  return DISC_OK;
}

void free_levels(disc_ctx* c) {
  for (int l = 0; l < DISC_MAX_LEVELS; ++l) {
    Level& v = c->lev[l];
    if (v.graph) cudaGraphExecDestroy(v.graph);
    if (v.loop) cudaGraphExecDestroy(v.loop);
    cudaFree(v.Im);
    cudaFree(v.Is);
    cudaFree(v.zs);
    cudaFree(v.m);
    cudaFree(v.r);
    cudaFree(v.u);
    cudaFree(v.t);
    cudaFree(v.hist);
    cudaFree(v.hsum);
    cudaFree(v.sd);
    cudaFree(v.ab);
    cudaFree(v.isab);
    cudaFree(v.dm);
    cudaFree(v.stamp);
    cudaFree(v.kbits);
    cudaFree(v.flist);
    cudaFree(v.cnt);
    v = Level{};
  }
  cudaFree(c->d_mwork);
  c->d_mwork = nullptr;
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
  a.u_is_dr = c->p.smooth_mode;
  a.nx = v.nx;
  a.ny = v.ny;
  a.nz = v.nz;
  a.hx = c->hx;
  a.hy = c->hy;
  a.hz = c->hz;
  a.var_floor = c->p.var_floor;
  a.force_mode = c->p.force_mode;
  a.norm_lo = v.norm_lo;
  a.norm_hi = v.norm_hi;
  return a;
}

// Mask-and-fill correction of level l for the current m (Algorithm A1 steps
// 1-3 with Eqs. 7-10): d = I'_s - m in v.dm.  stop: the level's stop flag, or
// NULL to run regardless.
// Inside a graph capture: the fill passes as a conditional WHILE node whose body
// (kFillPassesPerBody passes, captured on the side stream) runs again only while
// the last pass's front was not empty, so passes with nothing left to fill cost
// no launches (a pass after an empty front returns at entry).  The pass index
// lives on the device after cnt[passes].
constexpr int kFillPassesPerBody = 2;
cudaError_t queue_fill_loop(disc_ctx* c, Level& v, FillArgs f, size_t W) {
  f.next = v.cnt + c->p.fill_passes + 1;
  f.kbits = v.kbits;
  f.kwords = (long long)W;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(c->s, &cs, nullptr, &g, &deps, nullptr, &nd);
  if (e != cudaSuccess) return e;
  cudaGraphConditionalHandle h = 0;
  e = cudaGraphConditionalHandleCreate(&h, g, 0u, 0u);
  if (e != cudaSuccess) return e;
  f.cond = h;
  f.use_cond = 1;
  e = launch_fill_loop_start(f, c->s);       // pass 1 next; run the loop if anything is masked
  if (e != cudaSuccess) return e;
  e = cudaStreamGetCaptureInfo(c->s, &cs, nullptr, &g, &deps, nullptr, &nd);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &cp);
  if (e != cudaSuccess) return e;
  e = cudaStreamBeginCaptureToGraph(c->side, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                    cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t e1 = cudaSuccess;
  for (int k = 0; k < kFillPassesPerBody && e1 == cudaSuccess; ++k) e1 = launch_fill_pass(f, c->side);
  cudaGraph_t body = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(c->side, &body);
  if (e1 != cudaSuccess) return e1;
  if (e2 != cudaSuccess) return e2;
  // the capture of c->s continues after the loop node
  return cudaStreamUpdateCaptureDependencies(c->s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

cudaError_t queue_mask_fill(disc_ctx* c, int l, const int* stop) {
  Level& v = c->lev[l];
  cudaError_t e = cudaMemsetAsync(v.cnt, 0, (c->p.fill_passes + 1) * sizeof(int), c->s);
  if (e != cudaSuccess) return e;
  BoxArgs a = box_args(c, v);
  a.src = v.m;
  a.zs = v.zs;
  a.is = v.Is;
  a.sd = v.sd;
  a.out = v.dm;
  a.isab = v.isab;
  a.stamp = v.stamp;
  a.count = v.cnt;
  a.hu0 = c->mask_hu0;
  a.a_min = c->p.a_lo * c->mask_am;
  a.a_max = c->p.a_hi * c->mask_am;
  a.stop = stop;
  a.qscale = c->qs_m;
  a.inv_qscale = 1.0f / c->qs_m;
  e = box_launch(kModeMaskAB, a, v.pm, c->s);
  FillArgs f{};
  f.isab = v.isab;
  f.m = v.m;
  f.d = v.dm;
  f.stamp = v.stamp;
  f.cnt = v.cnt;
  f.passes = c->p.fill_passes;
  f.nwx = (v.nx + 31) / 32;
  f.list = v.flist;
  f.boff = v.flist + v.N;
  f.nfront = f.boff + fill_front_blocks(v.nx, v.ny, v.nz);
  const size_t W = (size_t)fill_words(v.nx, v.ny, v.nz);
  if (e == cudaSuccess) e = launch_fill_pack(v.stamp, v.kbits, v.nx, v.ny, v.nz, c->s);
  f.nx = v.nx;
  f.ny = v.ny;
  f.nz = v.nz;
  f.tx = (c->p.fill_t[0] - 1) / 2;
  f.ty = (c->p.fill_t[1] - 1) / 2;
  f.tz = (c->p.fill_t[2] - 1) / 2;
  f.inv_h = 1.0f / c->p.fill_h;
  f.stop = stop;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (e == cudaSuccess) e = cudaStreamIsCapturing(c->s, &cs);
  if (e == cudaSuccess && cs == cudaStreamCaptureStatusActive) return queue_fill_loop(c, v, f, W);
  for (int p = 1; p <= c->p.fill_passes && e == cudaSuccess; ++p) {
    f.pass = p;
    f.kin = v.kbits + ((p - 1) % 2) * W;
    f.kout = v.kbits + (p % 2) * W;
    e = launch_fill_pass(f, c->s);
  }
  return e;
}

// The masked iteration: mask and fill, force from d and m, Gaussian (+ warp), norm.
cudaError_t queue_masked(disc_ctx* c, int l, int n, const GaussArgs& g, const NormState& st) {
  Level& v = c->lev[l];
  ForceArgs fa{};
  fa.d = v.dm;
  fa.m = v.m;
  fa.r = v.r;
  fa.u = v.u;
  fa.partials = c->partials;
  fa.norm_lo = v.norm_lo;
  fa.norm_hi = v.norm_hi;
  fa.stop = c->d_stop + l;
  fa.nx = v.nx;
  fa.ny = v.ny;
  fa.nz = v.nz;
  fa.force_mode = c->p.force_mode;
  fa.u_is_dr = c->p.smooth_mode;
  const int blocks = force_blocks((int64_t)v.N, c->max_parts);
  for (int k = 0; k < n; ++k) {
    cudaError_t e = queue_mask_fill(c, l, c->d_stop + l);
    if (e == cudaSuccess) e = launch_force_dm(fa, blocks, c->s);
    if (e == cudaSuccess) e = gauss_launch(g, v.pb, c->s);
    if (e == cudaSuccess && v.sep_warp) e = launch_warp(v.Im, v.r, v.m, v.nx, v.ny, v.nz, c->d_stop + l, c->s);
    if (e == cudaSuccess) e = launch_norm_finalize(c->partials, blocks, st, c->s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// In-graph loop control: the norm kernel decrements *budget and sets `cond`.
struct LoopCond {
  int* budget;
  cudaGraphConditionalHandle cond;
};

// Queue `n` iterations of level l (box pass, Gaussian pass, norm) on c->s.
// With `loop`, the norm kernel also drives the loop graph's condition and the
// level-start warp is left to the caller.
cudaError_t queue_iterations(disc_ctx* c, int l, int n, const LoopCond* loop) {
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
  g.m = v.sep_warp ? nullptr : v.m;   // the xy pass also warps I_m for the next iteration
  g.add = c->p.smooth_mode ? v.r : nullptr;   // r <- r + G * dr (Sec. 2.1 order)
  g.stop = c->d_stop + l;
  g.nx = v.nx;
  g.ny = v.ny;
  g.nz = v.nz;
  g.R = c->R;
  std::memcpy(g.w, c->w, sizeof(c->w));
  NormState st{v.hist, v.hsum, c->d_iter + l, c->d_stop + l, v.hist_cap, c->p.stop_window, c->p.stop_eps};
  if (loop) {
    st.budget = loop->budget;
    st.cond = loop->cond;
    st.use_cond = 1;
  }
  const int nparts = (int)(v.pa.grid.x * v.pa.grid.y * v.pa.grid.z);
  // m for the field the first iteration starts from; later iterations get it
  // from the fused warp of the Gaussian xy pass
  if (!loop) {
    cudaError_t e0 = launch_warp(v.Im, v.r, v.m, v.nx, v.ny, v.nz, c->d_stop + l, c->s);
    if (e0 != cudaSuccess) return e0;
  }
  if (c->p.mask_mode) return queue_masked(c, l, n, g, st);
  for (int k = 0; k < n; ++k) {
    cudaError_t e;
    {
      NvtxRange r("disc moments, correction, force");
      e = box_launch(kModeIterate, a, v.pa, c->s);
    }
    if (e != cudaSuccess) return e;
    {
      NvtxRange r("disc Gaussian");
      e = gauss_launch(g, v.pb, c->s);
    }
    if (e != cudaSuccess) return e;
    if (v.sep_warp) {
      NvtxRange r("disc warp");
      e = launch_warp(v.Im, v.r, v.m, v.nx, v.ny, v.nz, c->d_stop + l, c->s);
      if (e != cudaSuccess) return e;
    }
    {
      NvtxRange r("disc norm");
      e = launch_norm_finalize(c->partials, nparts, st, c->s);
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Kernel nodes of a graph, child graphs included; kernels inside a
// conditional node's body (run a number of times decided on the device) are
// not counted.
long long graph_kernel_nodes(cudaGraph_t g) {
  size_t n = 0;
  if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  std::vector<cudaGraphNode_t> nodes(n);
  if (n > 0 && cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  long long k = 0;
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType t = cudaGraphNodeTypeEmpty;
    if (cudaGraphNodeGetType(nd, &t) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (t == cudaGraphNodeTypeKernel) {
      ++k;
    } else if (t == cudaGraphNodeTypeGraph) {
      cudaGraph_t child = nullptr;
      if (cudaGraphChildGraphNodeGetGraph(nd, &child) == cudaSuccess) k += graph_kernel_nodes(child);
      else cudaGetLastError();
    }
  }
  return k;
}

// The loop graph of level l: a conditional WHILE node whose body is one
// iteration; the body's norm kernel leaves the loop when the launch's budget
// of iterations is spent or the stop rule fires (Sec. 2.3), so a stopped level
// runs no further kernels.
cudaError_t build_loop_graph(disc_ctx* c, int l) {
  Level& v = c->lev[l];
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return e;
  cudaGraphConditionalHandle h = 0;
  e = cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault);
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp);
  if (e == cudaSuccess) {
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(c->s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const LoopCond lc{c->d_budget + l, h};
      const cudaError_t e1 = queue_iterations(c, l, 1, &lc);
      cudaGraph_t captured = nullptr;
      const cudaError_t e2 = cudaStreamEndCapture(c->s, &captured);
      e = e1 != cudaSuccess ? e1 : e2;
      if (e == cudaSuccess) v.loop_kernels = graph_kernel_nodes(body);
    }
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&v.loop, g, 0);
  if (e != cudaSuccess) v.loop = nullptr;
  cudaGraphDestroy(g);
  return e;
}

cudaError_t run_iterations(disc_ctx* c, int l, int n) {
  if (n <= 0) return cudaSuccess;
  Level& v = c->lev[l];
  char name[64];
  std::snprintf(name, sizeof(name), "disc level %d: %d iterations", l, n);
  NvtxRange range(name);
  if (!c->use_graphs) {
    c->launches = -1;                      // stream launches are not counted
    return queue_iterations(c, l, n, nullptr);
  }
  if (c->use_loop) {
    if (v.loop == nullptr) {
      const cudaError_t e = build_loop_graph(c, l);
      if (e != cudaSuccess) return e;
    }
    cudaError_t e = launch_warp(v.Im, v.r, v.m, v.nx, v.ny, v.nz, c->d_stop + l, c->s);
    if (e == cudaSuccess) e = launch_set_int(c->d_budget + l, n, c->s);
    if (e == cudaSuccess) e = cudaGraphLaunch(v.loop, c->s);
    // the body's kernels for each of the n iterations the budget allows (the
    // stop rule may end the level earlier)
    if (e == cudaSuccess && c->launches >= 0) c->launches += 2 + v.loop_kernels * n;
    return e;
  }
  if (v.graph == nullptr || v.graph_iters != n) {
    if (v.graph) {
      cudaGraphExecDestroy(v.graph);
      v.graph = nullptr;
    }
    cudaGraph_t gph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c->s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    e = queue_iterations(c, l, n, nullptr);
    cudaError_t e2 = cudaStreamEndCapture(c->s, &gph);
    if (e != cudaSuccess) {
      if (gph) cudaGraphDestroy(gph);
      return e;
    }
    if (e2 != cudaSuccess) return e2;
    v.graph_kernels = graph_kernel_nodes(gph);
    e = cudaGraphInstantiate(&v.graph, gph, 0);
    cudaGraphDestroy(gph);
    if (e != cudaSuccess) {
      v.graph = nullptr;
      return e;
    }
    v.graph_iters = n;
  }
  const cudaError_t e = cudaGraphLaunch(v.graph, c->s);
  if (e == cudaSuccess && c->launches >= 0) c->launches += v.graph_kernels;
  return e;
}

cudaError_t reset_level_counters(disc_ctx* c, int l) {
  cudaError_t e = cudaMemsetAsync(c->d_iter + l, 0, sizeof(int), c->s);
  if (e != cudaSuccess) return e;
  return cudaMemsetAsync(c->d_stop + l, 0, sizeof(int), c->s);
}

}  // namespace

namespace disc {

cudaError_t ctx_reset_level_counters(disc_ctx* c, int l, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(c->d_iter + l, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  return cudaMemsetAsync(c->d_stop + l, 0, sizeof(int), s);
}

cudaError_t ctx_reserve_partials(disc_ctx* c, int n) {
  if (n <= c->max_parts) return cudaSuccess;
  cudaError_t e = cudaStreamSynchronize(c->s);
  if (e != cudaSuccess) return e;
  cudaFree(c->partials);
  c->partials = nullptr;
  c->max_parts = 0;
  e = cudaMalloc(&c->partials, sizeof(float) * 2 * (size_t)n);
  if (e != cudaSuccess) return e;
  c->max_parts = n;
  for (int l = 0; l < DISC_MAX_LEVELS; ++l) {   // the context's own graphs hold the old buffer
    Level& v = c->lev[l];
    if (v.graph) cudaGraphExecDestroy(v.graph);
    if (v.loop) cudaGraphExecDestroy(v.loop);
    v.graph = nullptr;
    v.loop = nullptr;
    v.graph_iters = 0;
  }
  return cudaSuccess;
}

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
  a.zlen = v.pn.zlen;
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
  g.add = c->p.smooth_mode ? v.r : nullptr;
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
  return NormState{v.hist, v.hsum, c->d_iter + l, c->d_stop + l, v.hist_cap, c->p.stop_window, c->p.stop_eps};
}

// Queue up to `budget` iterations of the schedule on ctx->s, from the
// context's current level and iteration (finished levels are up-sampled).
cudaError_t ctx_advance(disc_ctx* ctx, long long budget, int* touched, int* ntouched, long long* queued) {
  const int L = ctx->L;
  int nt = 0;
  long long q = 0;
  while (true) {
    const int l = ctx->cur_level;
    const int total = ctx->p.iters[L - 1 - l];
    const int left = total - ctx->cur_iter;
    if (left > 0 && budget > 0) {
      const int n = (int)(left < budget ? left : budget);
      const cudaError_t e = run_iterations(ctx, l, n);
      if (e != cudaSuccess) return e;
      if (touched && (nt == 0 || touched[nt - 1] != l)) touched[nt++] = l;
      ctx->cur_iter += n;
      budget -= n;
      q += n;
    }
    if (ctx->cur_iter >= total && l > 0) {
      // level finished: up-sample the field to the next finer level (Algorithm A1)
      const Level& fine = ctx->lev[l - 1];
      cudaError_t e = launch_up2(ctx->lev[l].r, fine.r, fine.nx, fine.ny, fine.nz, ctx->s);
      if (e != cudaSuccess) return e;
      if (ctx->launches >= 0) ctx->launches += 1;
      e = reset_level_counters(ctx, l - 1);
      if (e != cudaSuccess) return e;
      ctx->cur_level = l - 1;
      ctx->cur_iter = 0;
      continue;
    }
    break;
  }
  if (ntouched) *ntouched = nt;
  if (queued) *queued = q;
  return cudaSuccess;
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
  p->mask_mode = 0;
  p->hu0_factor = 2.0f;
  p->a_lo = 0.5f;
  p->a_hi = 1.5f;
  p->fill_h = 50.0f;
  p->fill_t[0] = p->fill_t[1] = 7;
  p->fill_t[2] = 3;
  p->fill_passes = 32;
  p->smooth_mode = 0;
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
  const uint32_t sw = test_switches();
  ctx->use_graphs = (sw & DISC_SW_NO_GRAPH) == 0u;
  // the loop graph pays a few microseconds per iteration for its condition; it
  // is used where it saves work, when the stop rule can end a level early
  ctx->use_loop = p->stop_eps > 0.0f && (sw & DISC_SW_UNROLLED_GRAPH) == 0u;
  ctx->separate_warp = (sw & DISC_SW_SEPARATE_WARP) ? 1 : 0;
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  cudaError_t e = cudaStreamCreateWithFlags(&ctx->s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming);
  ctx->user = static_cast<cudaStream_t>(cuda_stream);   // NULL: the legacy default stream
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_iter, sizeof(int) * DISC_MAX_LEVELS);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_stop, sizeof(int) * (DISC_MAX_LEVELS + 1));
  if (e == cudaSuccess) ctx->d_err = ctx->d_stop + DISC_MAX_LEVELS;
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_budget, sizeof(int) * DISC_MAX_LEVELS);
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
  cudaFree(ctx->d_budget);
  cudaFree(ctx->d_scratch);
  cudaFree(ctx->d_maxabs);
  if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
  if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
  if (ctx->s) cudaStreamDestroy(ctx->s);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  cudaGetLastError();
  delete ctx;
  return DISC_OK;
}

disc_status disc_set_images(disc_ctx* ctx, const float* ct, const float* cbct, int32_t nx, int32_t ny,
                            int32_t nz, int mem_kind) {
  NvtxRange nvtx_range("disc_set_images");
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
  // scalars the captured iteration graphs hold by value (buffers are reused as they are)
  const float old_qs_m = ctx->qs_m, old_hu0 = ctx->mask_hu0, old_am = ctx->mask_am;
  if (!same) {
    free_levels(ctx);
    int max_parts = 1;
    for (int l = 0; l < L; ++l) {
      Level& v = ctx->lev[l];
      v.nx = dims[l][0];
      v.ny = dims[l][1];
      v.nz = dims[l][2];
      v.N = (size_t)v.nx * v.ny * v.nz;
      v.pa = box_plan_iter(v.nx, v.ny, v.nz, ctx->hx, ctx->hy, ctx->hz, ctx->num_sms, nullptr, nullptr, nullptr);
      v.pn = box_plan(kModeIterate, v.nx, v.ny, v.nz, ctx->hx, ctx->hy, ctx->hz, ctx->num_sms);
      v.pb = gauss_plan(v.nx, v.ny, v.nz, ctx->R, ctx->num_sms);
      v.sep_warp = ctx->separate_warp == 1;
      BoxPlan ps = box_plan(kModeStatic, v.nx, v.ny, v.nz, ctx->hx, ctx->hy, ctx->hz, ctx->num_sms);
      if (v.pa.grid.x == 0 || v.pb.grid.x == 0 || ps.grid.x == 0) {
        free_levels(ctx);
        return DISC_ERR_SHAPE;   // patch or radius too large for shared memory
      }
      const int np = (int)(v.pa.grid.x * v.pa.grid.y * v.pa.grid.z);
      const int nn = (int)(v.pn.grid.x * v.pn.grid.y * v.pn.grid.z);
      if (np > max_parts) max_parts = np;
      if (nn > max_parts) max_parts = nn;
      v.hist_cap = ctx->p.iters[L - 1 - l] > 0 ? ctx->p.iters[L - 1 - l] : 1;
      int lo = ctx->p.norm_planes[0], hi = ctx->p.norm_planes[1];
      for (int k = 0; k < l; ++k) {
        lo = (lo + 1) / 2;
        hi = (hi + 1) / 2;
      }
      v.norm_lo = lo;
      v.norm_hi = hi;
      // DISC_SW_FAULT_ALLOC: host-side fault injection, the first allocation
      // reports an out-of-memory error (tests the recovery of a context)
      cudaError_t e = (test_switches() & DISC_SW_FAULT_ALLOC) ? cudaErrorMemoryAllocation
                                                             : cudaMalloc(&v.Im, v.N * sizeof(float));
      if (e == cudaSuccess) e = cudaMalloc(&v.Is, v.N * sizeof(float));
      if (e == cudaSuccess) e = cudaMalloc(&v.zs, v.N * sizeof(float));
      if (e == cudaSuccess) e = cudaMalloc(&v.m, v.N * sizeof(float));
      if (e == cudaSuccess) e = cudaMalloc(&v.r, 3 * v.N * sizeof(float));
      if (e == cudaSuccess) e = cudaMalloc(&v.u, 3 * v.N * sizeof(float));
      if (e == cudaSuccess) e = cudaMalloc(&v.t, 3 * v.N * sizeof(float));
      if (e == cudaSuccess) e = cudaMalloc(&v.hist, v.hist_cap * sizeof(float));
      if (e == cudaSuccess) e = cudaMalloc(&v.hsum, 2 * (size_t)v.hist_cap * sizeof(double));
      if (e == cudaSuccess && ctx->p.mask_mode) {
        // the wide-tile mask pass on large levels (library buffers: aligned)
        v.pm = box_plan_wide_mode(kModeMaskAB, v.nx, v.ny, v.nz, ctx->hx, ctx->hy, ctx->hz, ctx->num_sms,
                                  nullptr, nullptr);
        if (v.pm.grid.x == 0) e = cudaErrorInvalidConfiguration;
        if (e == cudaSuccess) e = cudaMalloc(&v.sd, v.N * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&v.ab, 2 * v.N * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&v.isab, v.N * sizeof(float4));
        if (e == cudaSuccess) e = cudaMalloc(&v.dm, v.N * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&v.stamp, v.N * sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc(&v.kbits, 2 * sizeof(unsigned) * (size_t)fill_words(v.nx, v.ny, v.nz));
        if (e == cudaSuccess)
          e = cudaMalloc(&v.flist, sizeof(int) * (v.N + (size_t)fill_front_blocks(v.nx, v.ny, v.nz) + 1));
        if (e == cudaSuccess) e = cudaMalloc(&v.cnt, (ctx->p.fill_passes + 2) * sizeof(int));
      }
      if (e != cudaSuccess) {
        free_levels(ctx);
        return e == cudaErrorInvalidConfiguration ? DISC_ERR_SHAPE : fail(ctx, e);
      }
    }
    if (ctx->p.mask_mode) {
      cudaError_t e = cudaMalloc(&ctx->d_mwork, median_work_words() * sizeof(unsigned));
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
  }
  ctx->have_images = true;
  CK(enter(ctx));
  Level& f = ctx->lev[0];
  CK(memcpy_kind(f.Im, ct, f.N * sizeof(float), DISC_MEM_DEVICE, mem_kind, ctx->s));
  CK(memcpy_kind(f.Is, cbct, f.N * sizeof(float), DISC_MEM_DEVICE, mem_kind, ctx->s));
  if (ctx->p.global_shift)
    CK(launch_global_shift(f.Im, f.Is, f.Is, (int64_t)f.N, ctx->d_scratch, nullptr, ctx->s));
  else if (ctx->p.mask_mode)   // dHU for HU0 only: the shifted copy goes to scratch
    CK(launch_global_shift(f.Im, f.Is, f.m, (int64_t)f.N, ctx->d_scratch, nullptr, ctx->s));
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
  for (int i = 0; i < 2; ++i) {
    if (ctx->p.quant_max[i] > 0.0f) {                   // a caller's bound (a slab of a larger volume)
      if (ctx->p.quant_max[i] < mx[i]) return DISC_ERR_ARG;
      mx[i] = ctx->p.quant_max[i];
    }
  }
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
    a.sd_out = v.sd;                           // NULL unless the mask is on
    BoxPlan ps = box_plan(kModeStatic, v.nx, v.ny, v.nz, ctx->hx, ctx->hy, ctx->hz, ctx->num_sms);
    CK(box_launch(kModeStatic, a, ps, ctx->s));
  }
  if (ctx->p.mask_mode) {
    // a_m: median of STD(M)/STD(S) at the finest level with r = 0 (m = I_m), and
    // HU0 from the global shift dHU (reading R18)
    BoxArgs a = box_args(ctx, f);
    a.src = f.Im;
    a.zs = f.zs;
    a.sd = f.sd;
    a.a_out = f.ab;
    a.ratio_only = 1;
    a.qscale = ctx->qs_m;
    a.inv_qscale = 1.0f / ctx->qs_m;
    CK(box_launch(kModeMaskAB, a, f.pm, ctx->s));
    CK(launch_median(f.ab, (int64_t)f.N, ctx->d_mwork, ctx->s));
    unsigned res[9] = {};
    double dhu = 0.0;
    CK(cudaMemcpyAsync(res, ctx->d_mwork + median_work_words() - 9, sizeof(res), cudaMemcpyDeviceToHost,
                       ctx->s));
    CK(cudaMemcpyAsync(&dhu, ctx->d_scratch + 2 * kShiftBlocks, sizeof(double), cudaMemcpyDeviceToHost,
                       ctx->s));
    CK(cudaStreamSynchronize(ctx->s));
    float lo = 0.0f, hi = 0.0f;
    std::memcpy(&lo, &res[4], sizeof(float));
    std::memcpy(&hi, &res[8], sizeof(float));
    ctx->mask_am = res[0] > 0 ? (float)(0.5 * ((double)lo + (double)hi)) : 0.0f;
    ctx->mask_hu0 = ctx->p.hu0_factor * (float)std::fabs(dhu);
  }
  // the graphs of the previous images stay valid unless a scalar they captured
  // changed: the fixed-point scale of I_m or the mask thresholds
  if (same && (ctx->qs_m != old_qs_m || ctx->mask_hu0 != old_hu0 || ctx->mask_am != old_am)) {
    for (int l = 0; l < L; ++l) {
      if (ctx->lev[l].graph) cudaGraphExecDestroy(ctx->lev[l].graph);
      if (ctx->lev[l].loop) cudaGraphExecDestroy(ctx->lev[l].loop);
      ctx->lev[l].graph = nullptr;
      ctx->lev[l].loop = nullptr;
      ctx->lev[l].graph_iters = 0;
    }
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
  NvtxRange nvtx_range("disc_iterate");
  if (!ctx) return DISC_ERR_ARG;
  if (ctx->sticky != DISC_OK) return DISC_ERR_STATE;
  if (!ctx->have_images) return DISC_ERR_STATE;
  DeviceGuard guard(ctx->device);
  if (!guard.ok) return DISC_ERR_CUDA;
  CK(enter(ctx));
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
  CK(ctx_advance(ctx, budget, touched, &ntouched, nullptr));
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
  NvtxRange nvtx_range("disc_get_field");
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

}  // extern "C"

namespace {

// The warped CT m = I_m(x + r(x)) into v.m and the corrected CBCT I'_s into
// v.u (first N floats) at the current level, on ctx->s.
cudaError_t corrected_into_u(disc_ctx* ctx) {
  Level& v = ctx->lev[ctx->cur_level];
  cudaError_t e = launch_warp(v.Im, v.r, v.m, v.nx, v.ny, v.nz, nullptr, ctx->s);
  if (e != cudaSuccess) return e;
  if (ctx->p.mask_mode) {                  // I'_s = m + d of the masked correction
    e = queue_mask_fill(ctx, ctx->cur_level, nullptr);
    return e != cudaSuccess ? e : launch_add(v.m, v.dm, v.u, (int64_t)v.N, ctx->s);
  }
  BoxArgs a = box_args(ctx, v);
  a.src = v.m;
  a.zs = v.zs;
  a.r = v.r;
  a.out = v.u;
  a.qscale = ctx->qs_m;
  a.inv_qscale = 1.0f / ctx->qs_m;
  BoxPlan pc = box_plan(kModeCorrected, v.nx, v.ny, v.nz, ctx->hx, ctx->hy, ctx->hz, ctx->num_sms);
  return box_launch(kModeCorrected, a, pc, ctx->s);
}

}  // namespace

extern "C" {

disc_status disc_get_correction_means(disc_ctx* ctx, double* mean_a, double* mean_b, int64_t* count) {
  if (!ctx || (!mean_a && !mean_b && !count)) return DISC_ERR_ARG;
  if (ctx->sticky != DISC_OK) return DISC_ERR_STATE;
  if (!ctx->have_images) return DISC_ERR_STATE;
  DeviceGuard guard(ctx->device);
  if (!guard.ok) return DISC_ERR_CUDA;
  NvtxRange nvtx_range("disc_get_correction_means");
  CK(enter(ctx));
  Level& v = ctx->lev[ctx->cur_level];
  CK(launch_warp(v.Im, v.r, v.m, v.nx, v.ny, v.nz, nullptr, ctx->s));
  double* sums = nullptr;                     // sum a, sum b, count
  CK(cudaMallocAsync(&sums, 3 * sizeof(double), ctx->s));
  cudaError_t e = cudaSuccess;
  float* tmp = nullptr;
  if (ctx->p.mask_mode) {
    // the masked correction as an iteration computes it: a, b after the fill
    e = queue_mask_fill(ctx, ctx->cur_level, nullptr);
    if (e == cudaSuccess) e = launch_ab_sums(v.isab, v.stamp, (int64_t)v.N, sums, ctx->s);
  } else {
    // Eqs. 5-6 where a is defined: STD(S) of the level, then the mask pass with
    // thresholds that mask nothing but the voxels without STD(S)
    e = cudaMallocAsync(&tmp, v.N * (sizeof(float4) + 3 * sizeof(float) + sizeof(int)) + 64, ctx->s);
    float4* isab = reinterpret_cast<float4*>(tmp);
    float* sd = reinterpret_cast<float*>(isab + v.N);
    float* zs = sd + v.N;
    float* d = zs + v.N;
    int* stamp = reinterpret_cast<int*>(d + v.N);
    int* cnt = stamp + v.N;
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(int), ctx->s);
    BoxArgs a = box_args(ctx, v);
    a.src = v.Is;
    a.out = zs;
    a.sd_out = sd;
    a.qscale = ctx->qs_s;
    a.inv_qscale = 1.0f / ctx->qs_s;
    const BoxPlan ps = box_plan(kModeStatic, v.nx, v.ny, v.nz, ctx->hx, ctx->hy, ctx->hz, ctx->num_sms);
    if (e == cudaSuccess) e = box_launch(kModeStatic, a, ps, ctx->s);
    BoxArgs b = box_args(ctx, v);
    b.src = v.m;
    b.zs = zs;
    b.is = v.Is;
    b.sd = sd;
    b.out = d;
    b.isab = isab;
    b.stamp = stamp;
    b.count = cnt;
    b.hu0 = INFINITY;
    b.a_min = 0.0f;
    b.a_max = INFINITY;
    b.qscale = ctx->qs_m;
    b.inv_qscale = 1.0f / ctx->qs_m;
    const BoxPlan pm = box_plan_wide_mode(kModeMaskAB, v.nx, v.ny, v.nz, ctx->hx, ctx->hy, ctx->hz,
                                          ctx->num_sms, nullptr, nullptr);
    if (e == cudaSuccess) e = box_launch(kModeMaskAB, b, pm, ctx->s);
    if (e == cudaSuccess) e = launch_ab_sums(isab, stamp, (int64_t)v.N, sums, ctx->s);
  }
  double h[3] = {0.0, 0.0, 0.0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, ctx->s);
  if (tmp) {
    const cudaError_t ef = cudaFreeAsync(tmp, ctx->s);
    if (e == cudaSuccess) e = ef;
  }
  const cudaError_t ef = cudaFreeAsync(sums, ctx->s);
  if (e == cudaSuccess) e = ef;
  CK(e);
  CK_DEV(ctx);                                // synchronises
  if (mean_a) *mean_a = h[2] > 0.0 ? h[0] / h[2] : NAN;
  if (mean_b) *mean_b = h[2] > 0.0 ? h[1] / h[2] : NAN;
  if (count) *count = (int64_t)h[2];
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
  CK(corrected_into_u(ctx));
  CK(memcpy_kind(out, v.u, v.N * sizeof(float), mem_kind, DISC_MEM_DEVICE, ctx->s));
  if (mem_kind == DISC_MEM_HOST) CK_DEV(ctx);
  CK(leave(ctx));
  return DISC_OK;
}

disc_status disc_get_metrics(disc_ctx* ctx, int32_t bins, float sigma, float t_low, float t_high, double* nmi,
                             double* rmse_edge) {
  if (!ctx) return DISC_ERR_ARG;
  if (bins < 2 || bins > 128 || !(sigma > 0.0f) || std::ceil(3.0 * sigma) > 16) return DISC_ERR_ARG;
  if (ctx->sticky != DISC_OK) return DISC_ERR_STATE;
  if (!ctx->have_images) return DISC_ERR_STATE;
  DeviceGuard guard(ctx->device);
  CK(enter(ctx));
  Level& v = ctx->lev[ctx->cur_level];
  CK(corrected_into_u(ctx));
  const int64_t N = (int64_t)v.N;
  double* d = nullptr;   // nmi, rmse
  uint8_t* edges = nullptr;
  CK(cudaMallocAsync(reinterpret_cast<void**>(&d), 2 * sizeof(double), ctx->s));
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&edges), 2 * N, ctx->s);
  if (e == cudaSuccess) e = metric_nmi(v.m, v.u, N, bins, d, ctx->s);
  if (e == cudaSuccess) e = metric_canny(v.m, edges, v.nx, v.ny, v.nz, sigma, t_low, t_high, ctx->s);
  if (e == cudaSuccess) e = metric_canny(v.u, edges + N, v.nx, v.ny, v.nz, sigma, t_low, t_high, ctx->s);
  if (e == cudaSuccess) e = metric_edge_rmse(edges, edges + N, N, d + 1, ctx->s);
  double h[2] = {0.0, 0.0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, ctx->s);
  if (edges) cudaFreeAsync(edges, ctx->s);
  cudaFreeAsync(d, ctx->s);
  CK(e);
  CK_DEV(ctx);
  if (nmi) *nmi = h[0];
  if (rmse_edge) *rmse_edge = h[1];
  CK(leave(ctx));
  return DISC_OK;
}

disc_status disc_get_level_field(disc_ctx* ctx, int32_t level, float* out, int mem_kind) {
  if (!ctx || !out) return DISC_ERR_ARG;
  if (mem_kind != DISC_MEM_HOST && mem_kind != DISC_MEM_DEVICE) return DISC_ERR_ARG;
  if (ctx->sticky != DISC_OK) return DISC_ERR_STATE;
  if (!ctx->have_images) return DISC_ERR_STATE;
  if (level < 0 || level >= ctx->L) return DISC_ERR_ARG;
  DeviceGuard guard(ctx->device);
  CK(enter(ctx));
  const Level& v = ctx->lev[level];
  CK(memcpy_kind(out, v.r, 3 * v.N * sizeof(float), mem_kind, DISC_MEM_DEVICE, ctx->s));
  if (mem_kind == DISC_MEM_HOST) CK_DEV(ctx);
  CK(leave(ctx));
  return DISC_OK;
}

disc_status disc_ssd(disc_ctx* ctx, int32_t level, const float* r, double* loss, float* grad, int mem_kind) {
  if (!ctx || !r || (!loss && !grad)) return DISC_ERR_ARG;
  if (mem_kind != DISC_MEM_HOST && mem_kind != DISC_MEM_DEVICE) return DISC_ERR_ARG;
  if (ctx->sticky != DISC_OK) return DISC_ERR_STATE;
  if (!ctx->have_images) return DISC_ERR_STATE;
  if (level < 0 || level >= ctx->L) return DISC_ERR_ARG;
  DeviceGuard guard(ctx->device);
  if (!guard.ok) return DISC_ERR_CUDA;
  CK(enter(ctx));
  Level& v = ctx->lev[level];
  const size_t bytes = 3 * v.N * sizeof(float);
  // host fields go through the level's u and t buffers, which every iteration
  // rewrites before reading (its warp rebuilds m as well)
  const float* rd = r;
  if (mem_kind == DISC_MEM_HOST) {
    CK(memcpy_kind(v.u, r, bytes, DISC_MEM_DEVICE, DISC_MEM_HOST, ctx->s));
    rd = v.u;
  }
  float* gd = grad && mem_kind == DISC_MEM_HOST ? v.t : grad;
  double* dl = nullptr;
  if (loss) CK(cudaMallocAsync(&dl, sizeof(double), ctx->s));
  const int32_t patch[3] = {ctx->p.patch[0], ctx->p.patch[1], ctx->p.patch[2]};
  disc_status st = gd ? disc_k_ssd_grad(v.Im, v.zs, rd, gd, dl, v.nx, v.ny, v.nz, patch, ctx->qs_m,
                                        ctx->p.var_floor, ctx->s)
                      : disc_k_ssd_loss(v.Im, v.zs, rd, dl, v.nx, v.ny, v.nz, patch, ctx->qs_m, ctx->p.var_floor,
                                        ctx->s);
  if (st == DISC_OK && grad && mem_kind == DISC_MEM_HOST)
    CK(memcpy_kind(grad, gd, bytes, DISC_MEM_HOST, DISC_MEM_DEVICE, ctx->s));
  double lv = 0.0;
  if (st == DISC_OK && loss) CK(cudaMemcpyAsync(&lv, dl, sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
  if (dl) CK(cudaFreeAsync(dl, ctx->s));
  if (st != DISC_OK) {
    if (st == DISC_ERR_CUDA && ctx->sticky == DISC_OK) ctx->sticky = DISC_ERR_CUDA;
    return st;
  }
  if (loss || mem_kind == DISC_MEM_HOST) {
    CK_DEV(ctx);                              // synchronises the stream
    if (loss) *loss = lv;
  }
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

disc_status disc_get_launch_count(disc_ctx* ctx, int64_t* launches) {
  if (!ctx || !launches) return DISC_ERR_ARG;
  *launches = ctx->launches;
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

disc_status disc_get_norm_sums(disc_ctx* ctx, int32_t level, double* out, int32_t cap, int32_t* count) {
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
  if (n > 0) CK(cudaMemcpy(out, v.hsum, 2 * (size_t)n * sizeof(double), cudaMemcpyDeviceToHost));
  *count = n;
  return DISC_OK;
}

// ============================================================================
// Kernel-level entry points
// ============================================================================

disc_status disc_get_mask_constants(disc_ctx* ctx, float* hu0, float* a_m) {
  if (!ctx) return DISC_ERR_ARG;
  if (!ctx->have_images || !ctx->p.mask_mode) return DISC_ERR_STATE;
  if (hu0) *hu0 = ctx->mask_hu0;
  if (a_m) *a_m = ctx->mask_am;
  return DISC_OK;
}

disc_status disc_k_static_stats(const float* Is, float* zs, float* sd, int32_t nx, int32_t ny, int32_t nz,
                                const int32_t patch[3], float qscale, float var_floor, void* stream) {
  int h[3];
  disc_status st = kcheck(nx, ny, nz, patch, qscale, var_floor, h);
  if (st != DISC_OK) return st;
  if (!Is || !zs || zs == Is || (sd && (sd == Is || sd == zs))) return DISC_ERR_ARG;
  BoxArgs a = kargs(nx, ny, nz, h, qscale, var_floor);
  a.src = Is;
  a.out = zs;
  a.sd_out = sd;
  return klaunch(kModeStatic, a, (cudaStream_t)stream);
}

disc_status disc_k_ratio_median(const float* m, const float* zs, const float* sd, float* a_work,
                                double* median_out, int32_t nx, int32_t ny, int32_t nz, const int32_t patch[3],
                                float qscale, float var_floor, void* stream) {
  int h[3];
  disc_status st = kcheck(nx, ny, nz, patch, qscale, var_floor, h);
  if (st != DISC_OK) return st;
  if (!m || !zs || !sd || !a_work || !median_out) return DISC_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  BoxArgs a = kargs(nx, ny, nz, h, qscale, var_floor);
  a.src = m;
  a.zs = zs;
  a.sd = sd;
  a.a_out = a_work;
  a.ratio_only = 1;
  st = klaunch(kModeMaskAB, a, s);
  if (st != DISC_OK) return st;
  unsigned* work = nullptr;
  if (cudaMallocAsync(&work, median_work_words() * sizeof(unsigned), s) != cudaSuccess) {
    cudaGetLastError();
    return DISC_ERR_OOM;
  }
  cudaError_t e = launch_median(a_work, (int64_t)nx * ny * nz, work, s);
  if (e == cudaSuccess) e = launch_median_finish(work, median_out, s);
  cudaError_t e2 = cudaFreeAsync(work, s);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    cudaGetLastError();
    return DISC_ERR_CUDA;
  }
  return DISC_OK;
}

disc_status disc_k_correct_masked(const float* m, const float* Is, const float* zs, const float* sd, float* av,
                                  float* bv, float* d, int32_t* stamp, int32_t* remaining_out, int32_t nx,
                                  int32_t ny, int32_t nz, const int32_t patch[3], float qscale, float var_floor,
                                  float hu0, float a_min, float a_max, float fill_h, const int32_t fill_t[3],
                                  int32_t fill_passes, void* stream) {
  int h[3];
  disc_status st = kcheck(nx, ny, nz, patch, qscale, var_floor, h);
  if (st != DISC_OK) return st;
  if (!m || !Is || !zs || !sd || !av || !bv || !d || !stamp || !fill_t) return DISC_ERR_ARG;
  if (!(fill_h > 0.0f) || fill_passes < 1 || fill_passes > 1024 || !(hu0 >= 0.0f)) return DISC_ERR_ARG;
  for (int k = 0; k < 3; ++k)
    if (fill_t[k] < 1 || fill_t[k] > 15 || fill_t[k] % 2 == 0) return DISC_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t W = (size_t)fill_words(nx, ny, nz);
  const size_t N = (size_t)nx * ny * nz;
  const size_t FB = (size_t)fill_front_blocks(nx, ny, nz);
  // the counters [fill_passes + 1], two known-voxel bit masks [2][W], the front
  // list [N], its block offsets [FB] and length [1]
  keep_pool_memory();
  int* work = nullptr;
  if (cudaMallocAsync(&work, sizeof(int) * (fill_passes + 1 + 2 * W + N + FB + 1), s) != cudaSuccess) {
    cudaGetLastError();
    return DISC_ERR_OOM;
  }
  int* cnt = work;
  unsigned* kbits = reinterpret_cast<unsigned*>(work + fill_passes + 1);
  cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int) * (fill_passes + 1), s);
  BoxArgs a = kargs(nx, ny, nz, h, qscale, var_floor);
  a.src = m;
  a.zs = zs;
  a.is = Is;
  a.sd = sd;
  float4* isab = nullptr;   // the fill's working set, unpacked into av, bv at the end
  if (e == cudaSuccess) e = cudaMallocAsync(&isab, sizeof(float4) * N, s);
  a.out = d;
  a.isab = isab;
  a.stamp = stamp;
  a.count = cnt;
  a.hu0 = hu0;
  a.a_min = a_min;
  a.a_max = a_max;
  if (e == cudaSuccess) st = klaunch(kModeMaskAB, a, s);
  FillArgs f{};
  f.isab = isab;
  f.m = m;
  f.d = d;
  f.stamp = stamp;
  f.cnt = cnt;
  f.passes = fill_passes;
  f.nwx = (nx + 31) / 32;
  f.list = reinterpret_cast<int*>(kbits + 2 * W);
  f.boff = f.list + N;
  f.nfront = f.boff + FB;
  if (e == cudaSuccess && st == DISC_OK) e = launch_fill_pack(stamp, kbits, nx, ny, nz, s);
  f.nx = nx;
  f.ny = ny;
  f.nz = nz;
  f.tx = (fill_t[0] - 1) / 2;
  f.ty = (fill_t[1] - 1) / 2;
  f.tz = (fill_t[2] - 1) / 2;
  f.inv_h = 1.0f / fill_h;
  for (int p = 1; p <= fill_passes && e == cudaSuccess && st == DISC_OK; ++p) {
    f.pass = p;
    f.kin = kbits + ((p - 1) % 2) * W;
    f.kout = kbits + (p % 2) * W;
    e = launch_fill_pass(f, s);
  }
  if (e == cudaSuccess && st == DISC_OK && remaining_out) e = launch_fill_remaining(cnt, fill_passes, remaining_out, s);
  if (e == cudaSuccess && st == DISC_OK) e = launch_unpack_ab(isab, av, bv, (int64_t)N, s);
  if (isab) {
    const cudaError_t ef = cudaFreeAsync(isab, s);
    if (e == cudaSuccess) e = ef;
  }
  cudaError_t e2 = cudaFreeAsync(work, s);
  if (st != DISC_OK) return st;
  if (e != cudaSuccess || e2 != cudaSuccess) {
    cudaGetLastError();
    return DISC_ERR_CUDA;
  }
  return DISC_OK;
}

disc_status disc_k_force(const float* m, const float* d, const float* r, float* u, double* norms_out, int32_t nx,
                         int32_t ny, int32_t nz, int32_t force_mode, void* stream) {
  if (!m || !d || !r || !u || u == r) return DISC_ERR_ARG;
  if (force_mode != DISC_FORCE_THIRION && force_mode != DISC_FORCE_DOUBLE) return DISC_ERR_ARG;
  if (nx < 1 || ny < 1 || nz < 1 || (double)nx * ny * nz * 3.0 >= 2147483647.0) return DISC_ERR_SHAPE;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t N = (int64_t)nx * ny * nz;
  const int blocks = force_blocks(N, 148 * 8);
  float* parts = nullptr;
  if (cudaMallocAsync(&parts, sizeof(float) * 2 * blocks, s) != cudaSuccess) {
    cudaGetLastError();
    return DISC_ERR_OOM;
  }
  ForceArgs f{};
  f.d = d;
  f.m = m;
  f.r = r;
  f.u = u;
  f.partials = parts;
  f.nx = nx;
  f.ny = ny;
  f.nz = nz;
  f.force_mode = force_mode;
  cudaError_t e = launch_force_dm(f, blocks, s);
  if (e == cudaSuccess && norms_out) {
    e = launch_partials_sum(parts, blocks, 0, norms_out, s);
    if (e == cudaSuccess) e = launch_partials_sum(parts, blocks, 1, norms_out + 1, s);
  }
  cudaError_t e2 = cudaFreeAsync(parts, s);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    cudaGetLastError();
    return DISC_ERR_CUDA;
  }
  return DISC_OK;
}

disc_status disc_k_nmi(const float* a, const float* b, int64_t n, int32_t bins, double* nmi_out, void* stream) {
  if (!a || !b || !nmi_out || n < 1 || bins < 2 || bins > 128) return DISC_ERR_ARG;
  if (metric_nmi(a, b, n, bins, nmi_out, (cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    return DISC_ERR_CUDA;
  }
  return DISC_OK;
}

disc_status disc_k_canny(const float* img, uint8_t* edges, int32_t nx, int32_t ny, int32_t nz, float sigma,
                         float t_low, float t_high, void* stream) {
  if (!img || !edges || !(sigma > 0.0f) || std::ceil(3.0 * sigma) > 16) return DISC_ERR_ARG;
  if (!(t_low >= 0.0f) || !(t_high >= 0.0f)) return DISC_ERR_ARG;
  if (nx < 1 || ny < 1 || nz < 1 || (double)nx * ny * nz >= 2147483647.0) return DISC_ERR_SHAPE;
  if (metric_canny(img, edges, nx, ny, nz, sigma, t_low, t_high, (cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    return DISC_ERR_CUDA;
  }
  return DISC_OK;
}

disc_status disc_k_edge_rmse(const uint8_t* e1, const uint8_t* e2, int64_t n, double* out, void* stream) {
  if (!e1 || !e2 || !out || n < 1) return DISC_ERR_ARG;
  if (metric_edge_rmse(e1, e2, n, out, (cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    return DISC_ERR_CUDA;
  }
  return DISC_OK;
}

disc_status disc_k_check_error(void* stream) {
  int flag = 0;
  if (box_tma_error((cudaStream_t)stream, &flag) != cudaSuccess ||
      box_wide_error((cudaStream_t)stream, &flag) != cudaSuccess) {
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
  BoxPlan p = box_plan_iter(nx, ny, nz, h[0], h[1], h[2], sms, m_out, r, u);   // m_out NULL: pool memory, aligned
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
  BoxPlan p = box_plan_iter(nx, ny, nz, h[0], h[1], h[2], sms, m, r, u);
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
  keep_pool_memory();
  if (p.queue) CK(cudaMallocAsync(&t, sizeof(float) * 3 * (size_t)nx * ny * nz, s));
  g.t = t;
  cudaError_t e = gauss_launch(g, p, s);
  cudaError_t e2 = t ? cudaFreeAsync(t, s) : cudaSuccess;
  CK(e);
  CK(e2);
  return DISC_OK;
}

}  // extern "C"
