// Batched DISC: many CT/CBCT pairs of uneven size advanced together.
//
// Each pair keeps its own registration context (buffers, pyramid, CBCT patch
// statistics, field), but an iteration of all pairs is four launches in total
// instead of four per pair: the moment/force pass, the Gaussian xy pass, the
// Gaussian (with the next warp) and the norm, each over a work table
// that concatenates the CTA grids of every pair.  A level's iterations are
// captured once as a CUDA graph and replayed.  The moment/force launch is
// tuned per level at its first use: the z-chunk length of every pair's tiles
// and whether the launch has one CTA per work item or a persistent grid of one
// wave that strides over the table.  When every pair's level meets the
// bulk-tensor-copy conditions, the moment/force launch is the TMA-fed kernel,
// with each pair's four tensor maps in device memory.  Per pair the arithmetic
// is the one of the single-pair path, so each pair's field is bit-identical to
// a separate run.  With the mask of Eqs. 7-10 on, the pairs instead run their
// own single-pair schedules concurrently on their own streams (run_masked_batch).

#include <cstring>
#include <new>

#include "context.cuh"

using namespace disc;

struct disc_batch {
  disc_params p{};
  int device = 0;
  int num_sms = kNumSMs;
  cudaStream_t user = nullptr, s = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  int npairs = 0;
  disc_ctx* pair[kMaxBatch] = {};
  int L = 0, H = 0, R = 0;
  // work tables per level (kernel parameters of the batched launches)
  BoxBatch box[DISC_MAX_LEVELS];
  GaussBatch xy[DISC_MAX_LEVELS];
  GaussBatch zt[DISC_MAX_LEVELS];
  NormBatch norm[DISC_MAX_LEVELS];
  WarpBatch warp[DISC_MAX_LEVELS];
  int box_total[DISC_MAX_LEVELS] = {}, box_grid[DISC_MAX_LEVELS] = {}, zmult[DISC_MAX_LEVELS] = {};
  int xy_total[DISC_MAX_LEVELS] = {}, z_total[DISC_MAX_LEVELS] = {}, warp_total[DISC_MAX_LEVELS] = {};
  // the Gaussian z pass and the warp of the next iteration, tuned per level:
  // z chunk length (0: each pair's single-pair plan) and whether the warp runs
  // in the xy pass or as the z-marching warp kernel after it (table warpz)
  int gauss_zlen[DISC_MAX_LEVELS] = {};
  bool sep_warp[DISC_MAX_LEVELS] = {};
  WarpBatch warpz[DISC_MAX_LEVELS];
  int warpz_total[DISC_MAX_LEVELS] = {};
  bool ready[DISC_MAX_LEVELS] = {};
  // bulk-tensor-copy box pass at level l (every pair eligible): tensor maps of
  // all pairs in device memory, 4 per pair
  bool tma[DISC_MAX_LEVELS] = {};
  void* d_maps[DISC_MAX_LEVELS] = {};
  // the wide-tile box pass (32 x 32 tiles, balanced plane shares over all pairs)
  // where every pair's level allows it: its table, tensor maps and grid; used[l]
  // when the tuner (or a pin) chose it
  bool wide_ok[DISC_MAX_LEVELS] = {};
  bool wide[DISC_MAX_LEVELS] = {};
  WideBatch wtab[DISC_MAX_LEVELS];
  void* d_wmaps[DISC_MAX_LEVELS] = {};
  int wide_grid[DISC_MAX_LEVELS] = {};
  cudaGraphExec_t graph[DISC_MAX_LEVELS] = {};
  int graph_iters[DISC_MAX_LEVELS] = {};
  // tuning pinned by the caller (disc_batch_pin_tuning): z chunking and grid
  // (0: one CTA per work item) used instead of the autotuner's choice
  bool pinned[DISC_MAX_LEVELS] = {};
  int pin_zmult[DISC_MAX_LEVELS] = {}, pin_grid[DISC_MAX_LEVELS] = {};
  int cur_level = 0, cur_iter = 0;
  disc_status sticky = DISC_OK;
};

namespace {

disc_status bfail(disc_batch* b, cudaError_t e) {
  cudaGetLastError();
  if (e == cudaErrorMemoryAllocation) return DISC_ERR_OOM;
  if (b && b->sticky == DISC_OK) b->sticky = DISC_ERR_CUDA;
  return DISC_ERR_CUDA;
}

#define BCK(expr)                                \
  do {                                           \
    cudaError_t e_ = (expr);                     \
    if (e_ != cudaSuccess) return bfail(b, e_);  \
  } while (0)

cudaError_t benter(disc_batch* b) {
  cudaError_t e = cudaEventRecord(b->ev_in, b->user);
  if (e != cudaSuccess) return e;
  return cudaStreamWaitEvent(b->s, b->ev_in, 0);
}
cudaError_t bleave(disc_batch* b) {
  cudaError_t e = cudaEventRecord(b->ev_out, b->s);
  if (e != cudaSuccess) return e;
  return cudaStreamWaitEvent(b->user, b->ev_out, 0);
}

void drop_level(disc_batch* b, int l) {
  if (b->graph[l]) cudaGraphExecDestroy(b->graph[l]);
  b->graph[l] = nullptr;
  b->graph_iters[l] = 0;
  b->ready[l] = false;
}

bool all_images(const disc_batch* b) {
  for (int i = 0; i < b->npairs; ++i)
    if (!b->pair[i]->have_images) return false;
  return true;
}

// Box-pass work table of level l.  zmult > 0: every pair's single-pair z chunk
// lengthened zmult times; zmult < 0: chunks of -zmult planes (at least the
// single-pair chunk, so that no pair gets more CTAs than its partials hold).
void make_box_table(disc_batch* b, int l, int zmult, int* total) {
  BoxBatch& h = b->box[l];
  std::memset(&h, 0, sizeof(h));
  h.count = b->npairs;
  int off = 0;
  for (int i = 0; i < b->npairs; ++i) {
    const disc_ctx* c = b->pair[i];
    const Level& v = c->lev[l];
    BoxArgs a = ctx_box_args(c, l);
    a.zlen = zmult > 0 ? v.pn.zlen * zmult : (-zmult > v.pn.zlen ? -zmult : v.pn.zlen);
    if (a.zlen > v.nz) a.zlen = v.nz;
    h.args[i] = a;
    h.grid[i] = dim3(v.pn.grid.x, v.pn.grid.y, (v.nz + a.zlen - 1) / a.zlen);
    h.offset[i] = off;
    off += (int)(h.grid[i].x * h.grid[i].y * h.grid[i].z);
  }
  h.offset[b->npairs] = off;
  *total = off;
  // norm table: the same CTA counts
  NormBatch& n = b->norm[l];
  std::memset(&n, 0, sizeof(n));
  n.count = b->npairs;
  for (int i = 0; i < b->npairs; ++i) {
    n.partials[i] = b->pair[i]->partials;
    n.nparts[i] = h.offset[i + 1] - h.offset[i];
    n.st[i] = ctx_norm_state(b->pair[i], l);
  }
}

// Whether level l takes the bulk-tensor-copy box pass, and its tensor maps.
cudaError_t prepare_tma(disc_batch* b, int l) {
  b->tma[l] = false;
  for (int i = 0; i < b->npairs; ++i) {
    const disc_ctx* c = b->pair[i];
    const Level& v = c->lev[l];
    if (!box_tma_ok(kModeIterate, v.nx, v.ny, v.nz, b->H, b->H, b->H) ||
        !box_tma_aligned(kModeIterate, ctx_box_args(c, l)))
      return cudaSuccess;
  }
  alignas(128) unsigned char maps[kMaxBatch * 4 * kTmaMapBytes];
  for (int i = 0; i < b->npairs; ++i)
    if (!box_tma_encode(kModeIterate, ctx_box_args(b->pair[i], l), maps + i * 4 * kTmaMapBytes))
      return cudaSuccess;
  if (!b->d_maps[l]) {
    cudaError_t e = cudaMalloc(&b->d_maps[l], kMaxBatch * 4 * kTmaMapBytes);
    if (e != cudaSuccess) return e;
  }
  // pageable source: staged before the call returns; stream order publishes it
  cudaError_t e = cudaMemcpyAsync(b->d_maps[l], maps, b->npairs * 4 * kTmaMapBytes, cudaMemcpyHostToDevice, b->s);
  if (e != cudaSuccess) return e;
  b->tma[l] = true;
  return cudaSuccess;
}

// Whether every pair's level l can take the wide-tile box pass; if so its work
// table, tensor maps (device memory) and grid (one wave), and pair partials
// that hold one float2 per CTA of that grid.
cudaError_t prepare_wide(disc_batch* b, int l) {
  b->wide_ok[l] = false;
  for (int i = 0; i < b->npairs; ++i) {
    const Level& v = b->pair[i]->lev[l];
    if (!box_wide_ok(v.nx, v.ny, v.nz, b->H, b->H, b->H)) return cudaSuccess;
  }
  int tx = 0, ty = 0;
  box_wide_tile(&tx, &ty);
  const int occ = box_wide_occupancy(b->H);
  if (occ < 1) return cudaSuccess;
  const int grid = b->num_sms * occ;
  alignas(128) unsigned char maps[kMaxBatch * 2 * kTmaMapBytes];
  WideBatch& w = b->wtab[l];
  std::memset(&w, 0, sizeof(w));
  w.count = b->npairs;
  long long off = 0;
  for (int i = 0; i < b->npairs; ++i) {
    cudaError_t e = ctx_reserve_partials(b->pair[i], grid);
    if (e != cudaSuccess) return e;
    const Level& v = b->pair[i]->lev[l];
    w.args[i] = ctx_box_args(b->pair[i], l);
    if (!box_wide_encode(w.args[i], maps + i * 2 * kTmaMapBytes)) return cudaSuccess;
    w.tiles_x[i] = (v.nx + tx - 1) / tx;
    w.off[i] = off;
    off += (long long)w.tiles_x[i] * ((v.ny + ty - 1) / ty) * v.nz;
  }
  w.off[b->npairs] = off;
  if (!b->d_wmaps[l]) {
    cudaError_t e = cudaMalloc(&b->d_wmaps[l], kMaxBatch * 2 * kTmaMapBytes);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaMemcpyAsync(b->d_wmaps[l], maps, b->npairs * 2 * kTmaMapBytes, cudaMemcpyHostToDevice, b->s);
  if (e != cudaSuccess) return e;
  // pageable source: cudaMemcpyAsync has staged it when it returns; the stream
  // orders the copy before the launches
  b->wide_grid[l] = grid;
  b->wide_ok[l] = true;
  return cudaSuccess;
}

// Norm table of the wide launch: every pair adds one partial per CTA.
void make_wide_norm_table(disc_batch* b, int l, int grid) {
  NormBatch& n = b->norm[l];
  std::memset(&n, 0, sizeof(n));
  n.count = b->npairs;
  for (int i = 0; i < b->npairs; ++i) {
    n.partials[i] = b->pair[i]->partials;
    n.nparts[i] = grid;
    n.st[i] = ctx_norm_state(b->pair[i], l);
  }
}

// Gaussian z-pass table of level l (u -> t) with chunks of `zlen` planes (0:
// each pair's single-pair plan).
int make_z_table(disc_batch* b, int l, int zlen, GaussBatch& z) {
  std::memset(&z, 0, sizeof(z));
  z.count = b->npairs;
  int oz = 0;
  for (int i = 0; i < b->npairs; ++i) {
    const disc_ctx* c = b->pair[i];
    const Level& v = c->lev[l];
    GaussArgs g = ctx_gauss_args(c, l);
    g.r = g.t;
    g.add = nullptr;
    g.m = nullptr;
    if (zlen > 0) g.zlen = zlen < v.nz ? zlen : v.nz;
    z.args[i] = g;
    GaussPlan pl = v.pb;
    pl.zlen = g.zlen;
    dim3 gxy;
    gauss_grids(v.nx, v.ny, v.nz, pl, &gxy, &z.grid[i]);
    z.offset[i] = oz;
    oz += (int)(z.grid[i].x * z.grid[i].y * z.grid[i].z);
  }
  z.offset[b->npairs] = oz;
  return oz;
}

// Gaussian xy-pass table of level l (t -> r = add + G u; m = I_m(x + r) when
// `fused`), writing r and m to the given buffers (per pair; NULL: the pair's
// own).
int make_xy_table(disc_batch* b, int l, bool fused, GaussBatch& xy, float* const* r_to, float* const* m_to) {
  std::memset(&xy, 0, sizeof(xy));
  xy.count = b->npairs;
  int oxy = 0;
  for (int i = 0; i < b->npairs; ++i) {
    const disc_ctx* c = b->pair[i];
    const Level& v = c->lev[l];
    GaussArgs g = ctx_gauss_args(c, l);
    g.u = g.t;
    if (r_to) {
      g.r = r_to[i];
      if (g.add) g.add = r_to[i];
    }
    g.m = fused ? (m_to ? m_to[i] : v.m) : nullptr;
    xy.args[i] = g;
    dim3 gz;
    gauss_grids(v.nx, v.ny, v.nz, v.pb, &xy.grid[i], &gz);
    xy.offset[i] = oxy;
    oxy += (int)(xy.grid[i].x * xy.grid[i].y * xy.grid[i].z);
  }
  xy.offset[b->npairs] = oxy;
  return oxy;
}

// Batched z-marching warp table of level l (m from the given r per pair; NULL:
// the pair's own buffers).
int make_warpz_table(disc_batch* b, int l, WarpBatch& w, float* const* r_from, float* const* m_to) {
  std::memset(&w, 0, sizeof(w));
  w.count = b->npairs;
  int ow = 0;
  for (int i = 0; i < b->npairs; ++i) {
    const disc_ctx* c = b->pair[i];
    const Level& v = c->lev[l];
    w.offset[i] = ow;
    w.Im[i] = v.Im;
    w.r[i] = r_from ? r_from[i] : v.r;
    w.m[i] = m_to ? m_to[i] : v.m;
    w.nx[i] = v.nx;
    w.ny[i] = v.ny;
    w.nz[i] = v.nz;
    w.stop[i] = c->d_stop + l;
    ow += warp_z_blocks(v.nx, v.ny, v.nz);
  }
  w.offset[b->npairs] = ow;
  return ow;
}

void build_tables(disc_batch* b, int l) {
  WarpBatch& w = b->warp[l];
  std::memset(&w, 0, sizeof(w));
  w.count = b->npairs;
  int ow = 0;
  for (int i = 0; i < b->npairs; ++i) {
    const disc_ctx* c = b->pair[i];
    const Level& v = c->lev[l];
    w.offset[i] = ow;
    w.Im[i] = v.Im;
    w.r[i] = v.r;
    w.m[i] = v.m;
    w.nx[i] = v.nx;
    w.ny[i] = v.ny;
    w.nz[i] = v.nz;
    w.stop[i] = c->d_stop + l;
    ow += ((v.nx + kWarpBatchThreads - 1) / kWarpBatchThreads) * v.ny * v.nz;
  }
  w.offset[b->npairs] = ow;
  b->warp_total[l] = ow;
  b->gauss_zlen[l] = 0;
  b->sep_warp[l] = (test_switches() & DISC_SW_SEPARATE_WARP) != 0;
  b->z_total[l] = make_z_table(b, l, 0, b->zt[l]);
  b->xy_total[l] = make_xy_table(b, l, !b->sep_warp[l], b->xy[l], nullptr, nullptr);
  b->warpz_total[l] = make_warpz_table(b, l, b->warpz[l], nullptr, nullptr);
}

// Tuner of the Gaussian z pass and the warp placement at level l: the z pass
// for z chunks of each pair's plan, 16, 32 and 64 planes, then the xy pass with
// the warp fused, or followed by the z-marching warp kernel, timed on scratch
// copies of r and m so that the level's state is untouched (the z pass writes
// only t, which every iteration overwrites).  The default (fused, the pairs'
// plans) is replaced only by a choice at least 2% faster.  The test switches
// DISC_SW_SEPARATE_WARP / DISC_SW_FUSED_WARP fix the placement.
cudaError_t tune_gauss(disc_batch* b, int l) {
  size_t total = 0;
  for (int i = 0; i < b->npairs; ++i) total += 4 * b->pair[i]->lev[l].N;
  float* scratch = nullptr;
  cudaError_t e = cudaMallocAsync(&scratch, total * sizeof(float), b->s);
  if (e != cudaSuccess) return e;
  float* r_to[kMaxBatch];
  float* m_to[kMaxBatch];
  size_t off = 0;
  for (int i = 0; i < b->npairs; ++i) {
    const size_t N = b->pair[i]->lev[l].N;
    r_to[i] = scratch + off;
    m_to[i] = scratch + off + 3 * N;
    off += 4 * N;
  }
  e = cudaMemsetAsync(scratch, 0, total * sizeof(float), b->s);
  const uint32_t sw = test_switches();
  const int place_lo = (sw & DISC_SW_SEPARATE_WARP) ? 1 : 0;
  const int place_hi = (sw & DISC_SW_FUSED_WARP) ? 0 : 1;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  GaussBatch* zt_p = new (std::nothrow) GaussBatch;
  GaussBatch* xt_p = new (std::nothrow) GaussBatch;
  WarpBatch* wt_p = new (std::nothrow) WarpBatch;
  if (e == cudaSuccess && (!zt_p || !xt_p || !wt_p)) e = cudaErrorMemoryAllocation;
  GaussBatch& zt = *zt_p;
  GaussBatch& xt = *xt_p;
  WarpBatch& wt = *wt_p;
  const int zlens[4] = {0, 16, 32, 64};
  float best = 1e30f, deflt = 1e30f;
  int best_zlen = 0, best_sep = place_lo;
  for (int place = place_lo; place <= place_hi && e == cudaSuccess; ++place) {
    const int wtot = make_warpz_table(b, l, wt, r_to, m_to);
    const int xtot = make_xy_table(b, l, place == 0, xt, r_to, m_to);
    for (int zi = 0; zi < 4 && e == cudaSuccess; ++zi) {
      const int ztot = make_z_table(b, l, zlens[zi], zt);
      float ms = 0.0f;
      for (int k = 0; k < 4 && e == cudaSuccess; ++k) {   // one warm-up, three timed
        if (k == 1) e = cudaEventRecord(e0, b->s);
        if (e == cudaSuccess)
          e = gauss_launch_batch(xt, xtot, zt, ztot, b->R, place == 0, b->s);
        if (e == cudaSuccess && place == 1) e = launch_warp_z_batch(wt, wtot, b->s);
      }
      if (e == cudaSuccess) e = cudaEventRecord(e1, b->s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) break;
      if (place == place_lo && zi == 0) deflt = ms;
      if (ms < best) {
        best = ms;
        best_zlen = zlens[zi];
        best_sep = place;
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  delete zt_p;
  delete xt_p;
  delete wt_p;
  const cudaError_t ef = cudaFreeAsync(scratch, b->s);
  if (e == cudaSuccess) e = ef;
  if (e != cudaSuccess) return e;
  if (!(best < 0.98f * deflt)) {
    best_zlen = 0;
    best_sep = place_lo;
  }
  b->gauss_zlen[l] = best_zlen;
  b->sep_warp[l] = best_sep != 0;
  b->z_total[l] = make_z_table(b, l, best_zlen, b->zt[l]);
  b->xy_total[l] = make_xy_table(b, l, !b->sep_warp[l], b->xy[l], nullptr, nullptr);
  return cudaSuccess;
}

size_t box_smem(const disc_batch* b, int l) {
  return b->tma[l] ? box_tma_smem(kModeIterate, b->H) : box_fast_smem(kModeIterate, b->H);
}

cudaError_t launch_box(disc_batch* b, int l, int total, int grid) {
  if (b->wide[l]) return box_wide_launch_batch(b->wtab[l], b->d_wmaps[l], b->H, grid, b->s);
  if (b->tma[l]) return box_tma_launch_batch(b->box[l], b->d_maps[l], b->H, grid, b->s);
  return box_fast_launch_batch(b->box[l], b->H, total, grid, box_smem(b, l), b->s);
}

// Autotuner: time the batched box launch for each z-chunk multiplier and for a
// one-CTA-per-item or one-wave persistent grid; keep the fastest.  Runs on the
// level's current state: the box pass only writes u and its partials, which the
// next real iteration overwrites.
cudaError_t tune_level(disc_batch* b, int l) {
  const size_t smem = box_smem(b, l);
  const int occ = b->tma[l] ? box_tma_batch_occupancy(b->H, smem) : box_fast_occupancy(kModeIterate, b->H, smem);
  const int slots = b->num_sms * (occ < 1 ? 1 : occ);
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  b->wide[l] = false;
  if (b->pinned[l] && b->pin_zmult[l] == 0) {   // the caller's choice: the wide-tile pass
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!b->wide_ok[l]) return cudaErrorInvalidValue;
    const int g = b->pin_grid[l] > 0 && b->pin_grid[l] < b->wide_grid[l] ? b->pin_grid[l] : b->wide_grid[l];
    b->wide[l] = true;
    b->zmult[l] = 0;
    b->box_total[l] = (int)(b->wtab[l].off[b->npairs] < (1LL << 30) ? b->wtab[l].off[b->npairs] : (1LL << 30));
    b->box_grid[l] = g;
    make_wide_norm_table(b, l, g);
    return cudaSuccess;
  }
  if (b->pinned[l]) {                        // the caller's choice, untimed
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int total = 0;
    make_box_table(b, l, b->pin_zmult[l], &total);
    b->zmult[l] = b->pin_zmult[l];
    b->box_total[l] = total;
    b->box_grid[l] = b->pin_grid[l] > 0 && b->pin_grid[l] < total ? b->pin_grid[l] : total;
    return cudaSuccess;
  }
  float best = 1e30f;
  int best_mult = 1, best_grid = 0;
  // single-pair chunks, twice and four times longer, and common chunk lengths of
  // 32, 64 planes and whole columns (1 << 20: capped at each pair's depth)
  const int mults[6] = {1, 2, 4, -32, -64, -(1 << 20)};
  for (int mi = 0; mi < 6 && e == cudaSuccess; ++mi) {
    int total = 0;
    make_box_table(b, l, mults[mi], &total);
    const int grids[2] = {total, total < slots ? total : slots};
    for (int gi = 0; gi < 2 && e == cudaSuccess; ++gi) {
      if (gi == 1 && grids[1] == grids[0]) continue;
      e = launch_box(b, l, total, grids[gi]);   // warm-up
      if (e == cudaSuccess) e = cudaEventRecord(e0, b->s);
      for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = launch_box(b, l, total, grids[gi]);
      if (e == cudaSuccess) e = cudaEventRecord(e1, b->s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess && ms < best) {
        best = ms;
        best_mult = mults[mi];
        best_grid = grids[gi];
      }
    }
  }
  // the wide-tile pass over all pairs, one wave
  bool best_wide = false;
  if (e == cudaSuccess && b->wide_ok[l]) {
    b->wide[l] = true;
    const int g = b->wide_grid[l];
    e = launch_box(b, l, 0, g);               // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, b->s);
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = launch_box(b, l, 0, g);
    if (e == cudaSuccess) e = cudaEventRecord(e1, b->s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    // the wide launch changes the pass's resource use, which its three timed
    // launches alone do not show (the Gaussian passes that follow share the
    // SMs): it has to win by a clear margin
    if (e == cudaSuccess && ms < 0.9f * best) {
      best = ms;
      best_wide = true;
    }
    b->wide[l] = false;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  if (best_wide) {
    const long long P = b->wtab[l].off[b->npairs];
    b->wide[l] = true;
    b->zmult[l] = 0;
    b->box_total[l] = (int)(P < (1LL << 30) ? P : (1LL << 30));
    b->box_grid[l] = b->wide_grid[l];
    make_wide_norm_table(b, l, b->wide_grid[l]);
    return cudaSuccess;
  }
  int total = 0;
  make_box_table(b, l, best_mult, &total);
  b->zmult[l] = best_mult;
  b->box_total[l] = total;
  b->box_grid[l] = best_grid;
  return cudaSuccess;
}

cudaError_t queue_batch_iterations(disc_batch* b, int l, int n) {
  cudaError_t e = launch_warp_batch(b->warp[l], b->warp_total[l], b->s);
  for (int k = 0; k < n && e == cudaSuccess; ++k) {
    e = launch_box(b, l, b->box_total[l], b->box_grid[l]);
    if (e == cudaSuccess)
      e = gauss_launch_batch(b->xy[l], b->xy_total[l], b->zt[l], b->z_total[l], b->R, !b->sep_warp[l], b->s);
    if (e == cudaSuccess && b->sep_warp[l]) e = launch_warp_z_batch(b->warpz[l], b->warpz_total[l], b->s);
    if (e == cudaSuccess) e = launch_norm_finalize_batch(b->norm[l], b->npairs, b->s);
  }
  return e;
}

// The masked batch (Eqs. 7-10 on): the mask-and-fill step has a data-dependent
// number of fill passes per pair, which a shared work table cannot carry, so
// each pair runs its own single-pair schedule (captured graphs, the fill loop
// as a conditional node) on its own stream, and the pairs' streams run
// concurrently between one fork and one join on the batch stream.
cudaError_t run_masked_batch(disc_batch* b, long long budget, long long* queued) {
  cudaError_t e = cudaEventRecord(b->ev_in, b->s);
  long long q = 0;
  for (int i = 0; i < b->npairs && e == cudaSuccess; ++i) {
    disc_ctx* c = b->pair[i];
    e = cudaStreamWaitEvent(c->s, b->ev_in, 0);
    long long qi = 0;
    if (e == cudaSuccess) e = ctx_advance(c, budget, nullptr, nullptr, &qi);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_out, c->s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->s, c->ev_out, 0);
    q = qi;                                   // the same schedule for every pair
  }
  if (e != cudaSuccess) return e;
  b->cur_level = b->pair[0]->cur_level;
  b->cur_iter = b->pair[0]->cur_iter;
  *queued = q;
  return cudaSuccess;
}

cudaError_t run_batch_iterations(disc_batch* b, int l, int n) {
  if (n <= 0) return cudaSuccess;
  if (b->graph[l] == nullptr || b->graph_iters[l] != n) {
    if (b->graph[l]) {
      cudaGraphExecDestroy(b->graph[l]);
      b->graph[l] = nullptr;
    }
    cudaGraph_t gph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    e = queue_batch_iterations(b, l, n);
    cudaError_t e2 = cudaStreamEndCapture(b->s, &gph);
    if (e != cudaSuccess) {
      if (gph) cudaGraphDestroy(gph);
      return e;
    }
    if (e2 != cudaSuccess) return e2;
    e = cudaGraphInstantiate(&b->graph[l], gph, 0);
    cudaGraphDestroy(gph);
    if (e != cudaSuccess) {
      b->graph[l] = nullptr;
      return e;
    }
    b->graph_iters[l] = n;
  }
  return cudaGraphLaunch(b->graph[l], b->s);
}

}  // namespace

extern "C" {

disc_status disc_batch_create(const disc_params* p, int device, void* cuda_stream, int32_t npairs,
                              disc_batch** out) {
  if (!out || !p) return DISC_ERR_ARG;
  *out = nullptr;
  if (npairs < 1 || npairs > kMaxBatch) return DISC_ERR_ARG;
  // the batched kernels are specialised for cubic patches and Gaussian radius <= 8
  if (p->patch[0] != p->patch[1] || p->patch[1] != p->patch[2] || p->patch[0] < 3 || p->patch[0] > 15 ||
      p->patch[0] % 2 == 0)
    return DISC_ERR_ARG;
  if (p->levels < 1 || p->levels > DISC_MAX_LEVELS || !(p->gauss_sigma > 0.0f)) return DISC_ERR_ARG;
  const int R = gauss_radius(p->gauss_sigma, p->gauss_radius);
  if (R < 1 || R > 8) return DISC_ERR_ARG;
  disc_batch* b = new (std::nothrow) disc_batch();
  if (!b) return DISC_ERR_OOM;
  b->p = *p;
  b->device = device;
  b->npairs = npairs;
  b->L = p->levels;
  b->H = (p->patch[0] - 1) / 2;
  b->R = R;
  DeviceGuard guard(device);
  cudaError_t e = cudaStreamCreateWithFlags(&b->s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
  if (e == cudaSuccess) cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, device);
  b->user = static_cast<cudaStream_t>(cuda_stream);
  disc_status st = e == cudaSuccess ? DISC_OK : DISC_ERR_CUDA;
  for (int i = 0; i < npairs && st == DISC_OK; ++i) st = disc_create(p, device, b->s, &b->pair[i]);
  if (st != DISC_OK) {
    disc_batch_destroy(b);
    return st;
  }
  b->cur_level = b->L - 1;
  *out = b;
  return DISC_OK;
}

disc_status disc_batch_destroy(disc_batch* b) {
  if (!b) return DISC_OK;
  DeviceGuard guard(b->device);
  if (b->s) cudaStreamSynchronize(b->s);
  for (int l = 0; l < DISC_MAX_LEVELS; ++l) {
    if (b->graph[l]) cudaGraphExecDestroy(b->graph[l]);
    if (b->d_maps[l]) cudaFree(b->d_maps[l]);
    if (b->d_wmaps[l]) cudaFree(b->d_wmaps[l]);
  }
  for (int i = 0; i < b->npairs; ++i) disc_destroy(b->pair[i]);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->s) cudaStreamDestroy(b->s);
  cudaGetLastError();
  delete b;
  return DISC_OK;
}

disc_status disc_batch_set_images(disc_batch* b, int32_t pair, const float* ct, const float* cbct, int32_t nx,
                                  int32_t ny, int32_t nz, int mem_kind) {
  if (!b || pair < 0 || pair >= b->npairs) return DISC_ERR_ARG;
  if (b->sticky != DISC_OK) return DISC_ERR_STATE;
  if (b->cur_level != b->L - 1 || b->cur_iter != 0) return DISC_ERR_STATE;   // only before iterating
  if ((double)nx * ny * nz * 3.0 >= 2147483647.0) return DISC_ERR_SHAPE;
  DeviceGuard guard(b->device);
  BCK(benter(b));
  disc_status st = disc_set_images(b->pair[pair], ct, cbct, nx, ny, nz, mem_kind);
  if (st != DISC_OK) return st;
  for (int l = 0; l < DISC_MAX_LEVELS; ++l) drop_level(b, l);
  BCK(bleave(b));
  return DISC_OK;
}

disc_status disc_batch_restart(disc_batch* b) {
  if (!b) return DISC_ERR_ARG;
  if (b->sticky != DISC_OK) return DISC_ERR_STATE;
  if (!all_images(b)) return DISC_ERR_STATE;
  DeviceGuard guard(b->device);
  BCK(benter(b));
  const int lc = b->L - 1;
  for (int i = 0; i < b->npairs; ++i) {
    disc_ctx* c = b->pair[i];
    BCK(cudaMemsetAsync(c->lev[lc].r, 0, 3 * c->lev[lc].N * sizeof(float), b->s));
    for (int l = 0; l < b->L; ++l) BCK(ctx_reset_level_counters(c, l, b->s));
    c->cur_level = lc;
    c->cur_iter = 0;
  }
  b->cur_level = lc;
  b->cur_iter = 0;
  BCK(bleave(b));
  return DISC_OK;
}

disc_status disc_batch_iterate(disc_batch* b, int32_t max_iters, int32_t* iters_done) {
  NvtxRange nvtx_range("disc_batch_iterate");
  if (!b) return DISC_ERR_ARG;
  if (b->sticky != DISC_OK) return DISC_ERR_STATE;
  if (!all_images(b)) return DISC_ERR_STATE;
  DeviceGuard guard(b->device);
  BCK(benter(b));
  long long budget = max_iters < 0 ? (1LL << 40) : max_iters;
  int done = 0;
  if (b->p.mask_mode) {
    long long q = 0;
    BCK(run_masked_batch(b, budget, &q));
    if (iters_done) *iters_done = (int32_t)q;
    BCK(bleave(b));
    return DISC_OK;
  }
  while (true) {
    const int l = b->cur_level;
    const int total = b->p.iters[b->L - 1 - l];
    const int left = total - b->cur_iter;
    if (left > 0 && budget > 0) {
      if (!b->ready[l]) {
        BCK(prepare_tma(b, l));
        BCK(prepare_wide(b, l));
        build_tables(b, l);
        BCK(launch_warp_batch(b->warp[l], b->warp_total[l], b->s));     // m for the tuning launches
        BCK(tune_level(b, l));
        BCK(tune_gauss(b, l));
        b->ready[l] = true;
      }
      const int n = (int)(left < budget ? left : budget);
      BCK(run_batch_iterations(b, l, n));
      b->cur_iter += n;
      budget -= n;
      done += n;
      for (int i = 0; i < b->npairs; ++i) b->pair[i]->cur_iter = b->cur_iter;
    }
    if (b->cur_iter >= total && l > 0) {
      for (int i = 0; i < b->npairs; ++i) {
        disc_ctx* c = b->pair[i];
        const Level& fine = c->lev[l - 1];
        BCK(launch_up2(c->lev[l].r, fine.r, fine.nx, fine.ny, fine.nz, b->s));
        BCK(ctx_reset_level_counters(c, l - 1, b->s));
        c->cur_level = l - 1;
        c->cur_iter = 0;
      }
      b->cur_level = l - 1;
      b->cur_iter = 0;
      continue;
    }
    break;
  }
  if (iters_done) *iters_done = done;
  BCK(bleave(b));
  return DISC_OK;
}

disc_status disc_batch_get_field(disc_batch* b, int32_t pair, float* out, int mem_kind) {
  if (!b || pair < 0 || pair >= b->npairs) return DISC_ERR_ARG;
  if (b->sticky != DISC_OK) return DISC_ERR_STATE;
  DeviceGuard guard(b->device);
  BCK(benter(b));
  disc_status st = disc_get_field(b->pair[pair], out, mem_kind);
  if (st != DISC_OK) return st;
  BCK(bleave(b));
  return DISC_OK;
}

disc_status disc_batch_get_tuning(disc_batch* b, int32_t level, int32_t* items, int32_t* grid,
                                  int32_t* zmult) {
  if (!b || level < 0 || level >= b->L) return DISC_ERR_ARG;
  if (!b->ready[level]) return DISC_ERR_STATE;
  if (items) *items = b->box_total[level];
  if (grid) *grid = b->box_grid[level];
  if (zmult) *zmult = b->zmult[level];
  return DISC_OK;
}

disc_status disc_batch_get_box_path(disc_batch* b, int32_t level, int32_t* tma) {
  if (!b || !tma || level < 0 || level >= b->L) return DISC_ERR_ARG;
  if (!b->ready[level]) return DISC_ERR_STATE;
  *tma = b->wide[level] ? 2 : (b->tma[level] ? 1 : 0);
  return DISC_OK;
}

disc_status disc_batch_get_gauss_tuning(disc_batch* b, int32_t level, int32_t* zlen, int32_t* separate_warp) {
  if (!b || level < 0 || level >= b->L) return DISC_ERR_ARG;
  if (!b->ready[level]) return DISC_ERR_STATE;
  if (zlen) *zlen = b->gauss_zlen[level];
  if (separate_warp) *separate_warp = b->sep_warp[level] ? 1 : 0;
  return DISC_OK;
}

disc_status disc_batch_pin_tuning(disc_batch* b, int32_t level, int32_t zmult, int32_t grid) {
  if (!b || level < 0 || level >= b->L) return DISC_ERR_ARG;
  if (grid < 0) return DISC_ERR_ARG;
  if (b->sticky != DISC_OK) return DISC_ERR_STATE;
  DeviceGuard guard(b->device);
  BCK(cudaStreamSynchronize(b->s));          // the level's graph may be in flight
  drop_level(b, level);                      // re-planned at the level's next iteration
  b->pinned[level] = true;
  b->pin_zmult[level] = zmult;
  b->pin_grid[level] = grid;
  return DISC_OK;
}

}  // extern "C"
