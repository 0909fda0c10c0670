// Internal declarations shared by the translation units of libdisc.so.
// Nothing here is part of the public ABI (include/disc.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "disc.h"

namespace disc {

// Test switches (disc_set_test_switches): one atomic word, set from the
// environment once at load and by the ABI call afterwards.
uint32_t test_switches();

// Bounds-checked build (compiled with -DDISC_BOUNDS_CHECK; the memory-safety
// check that stands in for a sanitizer): the per-iteration kernels test every
// global index against the extent of its buffer before the access.  An index
// out of range is not accessed (a load reads 0, a store is dropped) and is
// counted in a device-wide word that disc_bounds_violations reads; nothing
// traps.  In the normal build the test compiles to nothing.
#ifdef DISC_BOUNDS_CHECK
extern __device__ unsigned long long g_bounds_violations;
__device__ __forceinline__ bool index_ok(long long i, long long n) {
  if (i >= 0 && i < n) return true;
  atomicAdd(&g_bounds_violations, 1ull);
  return false;
}
#define DISC_IN(i, n) ::disc::index_ok((long long)(i), (long long)(n))
#else
#define DISC_IN(i, n) true
#endif
// p[i] of a buffer of n elements (read-only path), and p[i] = v, under that test.
template <typename T>
__device__ __forceinline__ T ldg_in(const T* p, long long i, long long n) {
  return DISC_IN(i, n) ? __ldg(p + i) : T{};
}
template <typename T>
__device__ __forceinline__ void st_in(T* p, long long i, long long n, T v) {
  if (DISC_IN(i, n)) p[i] = v;
}
// The same with the element given by its address p inside the buffer that
// starts at base (the index is formed only by the checked build).
template <typename T>
__device__ __forceinline__ T ldg_at(const T* p, const T* base, long long n) {
  return DISC_IN(p - base, n) ? __ldg(p) : T{};
}
template <typename T>
__device__ __forceinline__ void st_at(T* p, const T* base, long long n, T v) {
  if (DISC_IN(p - base, n)) *p = v;
}
// The same for data read or written once: streaming loads and stores (evicted
// first from L2, so that they do not push out data the kernel reuses).
template <typename T>
__device__ __forceinline__ T ldcs_in(const T* p, long long i, long long n) {
  return DISC_IN(i, n) ? __ldcs(p + i) : T{};
}
template <typename T>
__device__ __forceinline__ void stcs_in(T* p, long long i, long long n, T v) {
  if (DISC_IN(i, n)) __stcs(p + i, v);
}

constexpr int kThreads = 256;          // threads per CTA of every z-marching kernel
constexpr int kNumSMs = 148;           // B300: 2 dies x 74 SMs (queried at run time too)

// ----------------------------------------------------------------------------
// Index helpers
// ----------------------------------------------------------------------------
__host__ __device__ __forceinline__ size_t vix(int x, int y, int z, int nx, int ny) {
  return ((size_t)z * (size_t)ny + (size_t)y) * (size_t)nx + (size_t)x;
}

// Number of in-volume positions of the window [c-h, c+h] on an axis of n voxels
// (the truncated patch of the moment statistics, Eq. 3).
__host__ __device__ __forceinline__ int box_count(int c, int n, int h) {
  int lo = c - h < 0 ? 0 : c - h;
  int hi = c + h > n - 1 ? n - 1 : c + h;
  return hi - lo + 1;
}

// ----------------------------------------------------------------------------
// Patch-moment (box) kernels, box_pass.cu
// ----------------------------------------------------------------------------
enum BoxMode : int {
  kModeStatic = 0,     // zs = (I_s - E(S)) / STD(S)
  kModeIterate = 1,    // moments of m, correction, force, u = r + dr, norms
  kModeCorrected = 2,  // moments of m, I'_s written out
  kModeSsdLoss = 3,    // moments of m, per-CTA partial sum of (m - I'_s)^2
  kModeSsdAdjoint = 4, // moments of m, per-voxel adjoint coefficients (A, B, C, D)
  kModeMaskAB = 5      // moments of m: a, b of Eqs. 5-6, the mask xi of Eq. 7, d = I'_s - m
};

struct BoxArgs {
  const float* src;     // kModeStatic: I_s; otherwise the warped CT m = I_m(x + r)
  const float* zs;      // CBCT normalised patch value (all modes but kModeStatic)
  const float* r;       // field [3][N] (kModeIterate)
  float* out;           // kModeStatic: zs; kModeIterate: u [3][N]; kModeCorrected: I'_s;
                        // kModeSsdAdjoint: [4][N] (A, B, C, D)
  float* f_tap;         // optional (kModeIterate): I'_s - m
  float* partials;      // per-CTA float[2] (kModeIterate: sum|dr|, sum|r|; kModeSsdLoss: loss)
  int norm_lo, norm_hi; // kModeIterate: only planes [norm_lo, norm_hi) enter sum|dr|, sum|r|
                        // (all planes when norm_hi <= norm_lo, as zero-initialised)
  const int* stop;      // device flag: when non-zero the kernel returns at once
  int nx, ny, nz;
  int hx, hy, hz;       // patch half sizes
  float qscale, inv_qscale, var_floor;
  int force_mode;
  int zlen;             // output planes per CTA (z chunk)
  int* err;             // device error word (bit 0: a bulk-copy wait timed out); NULL: the library's own
  float* sd_out;        // optional (kModeStatic): STD(S) per voxel
  // kModeMaskAB (Eqs. 5-7): is = I_s, sd = STD(S); out = d = I'_s - m.  Outputs a, b,
  // stamp (0 where xi = 0, -1 where xi = 1) and the number of xi = 1 voxels (added to *count).
  // ratio_only: write only a = STD(M)/STD(S) (-1 where undefined) into a_out.
  const float* is;
  const float* sd;
  float* a_out;         // ratio_only: a per voxel (planar)
  float* b_out;
  float4* isab;         // kModeMaskAB: (I_s, a, b, 0) per voxel, the fill's working set
  int* stamp;
  int* count;
  float hu0, a_min, a_max;
  int ratio_only;
  int u_is_dr;          // kModeIterate: write u = dr instead of r + dr (smoothing of dr, Sec. 2.1)
  // test of the bounded waits (bulk-copy-fed pass only): bytes the first copy group
  // of a CTA is armed for beyond what its copies deliver, so that its wait gives up
  uint32_t stall_tx;
};

struct BoxPlan {
  dim3 grid;
  size_t smem;
  int zlen;
  int tx, ty;
  bool fast;            // cubic-patch kernel specialised on the half size (box_fast.cu)
  bool tma;             // the same kernel fed by bulk tensor copies (box_tma.cu)
  bool wide = false;    // iteration mode on wide tiles (box_wide.cu): grid.x CTAs share
                        // the volume's (tile, plane) pairs evenly
};

// Work table of a batched launch over many volumes (pairs): volume p owns the
// work items offset[p] .. offset[p+1]-1, which are the CTAs of its own grid.
// Tables are passed by value as kernel parameters (constant bank).
constexpr int kMaxBatch = 64;
struct BoxBatch {
  int count;
  int offset[kMaxBatch + 1];
  dim3 grid[kMaxBatch];
  BoxArgs args[kMaxBatch];
};

// Specialised cubic-patch path (box_fast.cu)
cudaError_t box_fast_launch_batch(const BoxBatch& bt, int h, int total, int grid, size_t smem,
                                  cudaStream_t s);
bool box_fast_ok(int nx, int ny, int nz, int hx, int hy, int hz);
size_t box_fast_smem(int mode, int h);
int box_fast_occupancy(int mode, int h, size_t smem);
cudaError_t box_fast_launch(int mode, const BoxArgs& a, const BoxPlan& p, cudaStream_t s);

// Bulk-tensor-copy path (box_tma.cu): usable when box_tma_ok (cubic patch, nx a
// multiple of 4, extents at least one staging box) and, per launch, when the
// buffers are 16-byte aligned (box_tma_aligned); the DISC_SW_NO_TMA test switch
// turns it off.
bool box_tma_ok(int mode, int nx, int ny, int nz, int hx, int hy, int hz);
bool box_tma_aligned(int mode, const BoxArgs& a);
size_t box_tma_smem(int mode, int h);
int box_tma_occupancy(int mode, int h, size_t smem);
cudaError_t box_tma_launch(int mode, const BoxArgs& a, const BoxPlan& p, cudaStream_t s);
// Reads (synchronising s) and clears the library's own error word into *flag.
cudaError_t box_tma_error(cudaStream_t s, int* flag);
// Batched iteration-mode launch: the tensor maps of volume p are maps[4p .. 4p+3]
// (kTmaMapBytes each, in device memory), written by box_tma_encode on the host.
constexpr size_t kTmaMapBytes = 128;
bool box_tma_encode(int mode, const BoxArgs& a, void* maps /* 4 x kTmaMapBytes, 64-byte aligned */);
int box_tma_batch_occupancy(int h, size_t smem);
cudaError_t box_tma_launch_batch(const BoxBatch& bt, const void* maps, int h, int grid, cudaStream_t s);

// Plan a launch (grid, z chunk, dynamic shared memory) for a volume and patch.
BoxPlan box_plan(int mode, int nx, int ny, int nz, int hx, int hy, int hz, int num_sms);
// Iteration-mode plan: the wide-tile pass (box_wide.cu) when the patch is cubic,
// the bulk-copy conditions hold, the warped image src, the field r and the
// output u are 16-byte aligned (NULL = library-owned buffers, which are) and
// the volume gives each CTA of its wave at least kWideMinPlanes planes; else
// box_plan's.
constexpr int kWideMinPlanes = 16;
// The mask mode's wide pass writes more per voxel (a, b, d, stamp) and won only
// where each CTA marches many planes: 4.1184 against 4.2238 s per masked
// 512x512x256 schedule, but 326.7 against 321.9 ms per 256x256x128 one (about
// 28 planes per CTA at its finest level).
constexpr int kWideMinPlanesMask = 64;
BoxPlan box_plan_iter(int nx, int ny, int nz, int hx, int hy, int hz, int num_sms, const float* src,
                      const float* r, const float* u);
// The same choice for the SSD adjoint pass (kModeSsdAdjoint) and the mask pass
// (kModeMaskAB, at least kWideMinPlanesMask planes per CTA): src the warped
// image, out the pass's first output buffer (the library's buffers are aligned;
// NULL is accepted).
BoxPlan box_plan_wide_mode(int mode, int nx, int ny, int nz, int hx, int hy, int hz, int num_sms,
                           const float* src, const float* out);
bool box_wide_ok(int nx, int ny, int nz, int hx, int hy, int hz);
size_t box_wide_smem(int h);
int box_wide_occupancy(int h);
void box_wide_tile(int* tx, int* ty);
// mode: kModeIterate, kModeSsdAdjoint or kModeMaskAB
cudaError_t box_wide_launch(int mode, const BoxArgs& a, const BoxPlan& p, cudaStream_t s);
// Reads (synchronising s) and clears the wide pass's own error word, OR-ing it into *flag.
cudaError_t box_wide_error(cudaStream_t s, int* flag);
// Batched wide-tile launch over many volumes: volume p owns planes [off[p],
// off[p + 1]) of the sequence of every volume's (tile, plane) pairs (tiles_x[p]
// tiles per row, args[p].nz planes per tile column); its two tensor maps are
// maps[2p], maps[2p + 1] (kTmaMapBytes each, written by box_wide_encode).
// args[p].partials needs one float2 per CTA of the launch.
struct WideBatch {
  int count;
  long long off[kMaxBatch + 1];
  int tiles_x[kMaxBatch];
  BoxArgs args[kMaxBatch];
};
bool box_wide_encode(const BoxArgs& a, void* maps /* 2 x kTmaMapBytes, 64-byte aligned */);
cudaError_t box_wide_launch_batch(const WideBatch& wb, const void* maps, int h, int grid, cudaStream_t s);
cudaError_t box_launch(int mode, const BoxArgs& a, const BoxPlan& plan, cudaStream_t s);

// Trilinear warp m = I_m(x + r(x)), warp.cu
cudaError_t launch_warp(const float* Im, const float* r, float* m, int nx, int ny, int nz, const int* stop,
                        cudaStream_t s);

// ----------------------------------------------------------------------------
// Gaussian pass, gauss.cu
// ----------------------------------------------------------------------------
struct GaussArgs {
  const float* u;       // [3][N] input field
  float* r;             // [3][N] smoothed field
  float* t;             // [3][N] scratch: the z-filtered field (split kernels)
  const float* Im;      // moving image, for the fused warp (may be NULL)
  float* m;             // if non-NULL: m = I_m(x + r(x)) is written too
  const int* stop;
  int nx, ny, nz;
  int R;
  int zlen;
  int box_sum;          // 1: plain truncated sums (no renormalisation at the borders)
  const float* add;     // optional [3][N]: the last pass writes r = add + G * u (add may be r itself)
  float w[2 * DISC_MAX_GAUSS_RADIUS + 1];   // normalised taps (sum 1), or all 1 for box sums
};
struct GaussPlan {
  dim3 grid;
  size_t smem;
  int zlen;
  bool queue;           // register-queue kernel (radius 1..8) or the generic one
};
struct GaussBatch {
  int count;
  int offset[kMaxBatch + 1];
  dim3 grid[kMaxBatch];
  GaussArgs args[kMaxBatch];
};
// Batched Gaussian passes over many volumes (gauss.cu): the z pass (u -> t) and
// the xy pass (t -> r = add + G u, and m when warp) with one launch each.  Work
// items follow each volume's own grids (xy: tiles x planes; z: column blocks x
// rows x chunks).
cudaError_t gauss_launch_batch(const GaussBatch& xy, int xy_total, const GaussBatch& z, int z_total,
                               int R, bool warp, cudaStream_t s);
void gauss_grids(int nx, int ny, int nz, const GaussPlan& p, dim3* xy, dim3* z);

int gauss_radius(float sigma, int radius);
void gauss_taps(float sigma, int R, float* w);
GaussPlan gauss_plan(int nx, int ny, int nz, int R, int num_sms);
cudaError_t gauss_launch(const GaussArgs& a, const GaussPlan& plan, cudaStream_t s);

// ----------------------------------------------------------------------------
// Differentiable form, ssd.cu
// ----------------------------------------------------------------------------
// grad = (D + S_A + m S_B - S_C) * dI_m/dp at p = x + r(x): the last step of the
// adjoint of the SSD loss (D, and the patch sums S of the coefficients A, B, C).
cudaError_t launch_ssd_final(const float* Im, const float* r, const float* m, const float* D,
                             const float* S, float* grad, int nx, int ny, int nz, cudaStream_t s);

// ----------------------------------------------------------------------------
// Mask and fill of a, b (Eqs. 7-10), mask.cu
// ----------------------------------------------------------------------------
struct FillArgs {
  float4* isab;         // (I_s, a, b, 0) per voxel: known a, b in, filled a, b out
  const float* m;       // I_m^(k)
  float* d;             // I'_s - m, written where a voxel is filled
  int* stamp;           // 0: xi = 0; p: filled by pass p; -1: not yet
  const unsigned* kin;  // known before this pass: bit masks, fill_words() words
  unsigned* kout;       // known after it (this pass writes it)
  int nwx;              // words per row, (nx + 31) / 32
  int* list;            // [N] the front of this pass, in voxel order
  int* boff;            // [fill_front_blocks] front counts, then offsets, per block of mask words
  int* nfront;          // [1] length of the list
  int* cnt;             // [passes + 1]: cnt[0] masked voxels (from the mask pass), cnt[p] filled by pass p
  int passes;           // passes of this fill
  int nx, ny, nz;
  int tx, ty, tz;       // half sizes of T
  float inv_h;          // 1 / h of Eq. 10
  int pass;             // 1, 2, ...
  const int* stop;
  // Device-driven passes (the body of a graph loop): when `next` is set, the
  // pass index is read from *next (the pass the next count kernel runs; the
  // scan kernel advances it) and kin, kout are picked from the pair `kbits`
  // ([2][kwords]) by its parity, in place of `pass`, `kin` and `kout`; with
  // use_cond the scan kernel also sets `cond` to continue while the front it
  // counted is not empty and passes remain.
  int* next;
  unsigned* kbits;
  long long kwords;
  cudaGraphConditionalHandle cond;
  int use_cond;
};
// One fill pass: the dilation of the known mask kin into kout, then the voxels
// of kout not in kin.  Before pass 1, launch_fill_pack sets kin from the stamps.
cudaError_t launch_fill_pass(const FillArgs& f, cudaStream_t s);
// Start of device-driven passes: *next = 1, and `cond` (the loop around the
// passes) set to run them unless the level has stopped, nothing is masked
// (cnt[0] = 0) or passes = 0.
cudaError_t launch_fill_loop_start(const FillArgs& f, cudaStream_t s);
// out[0..2] = sum of a, sum of b and the number of voxels with stamp >= 0.
cudaError_t launch_ab_sums(const float4* isab, const int* stamp, int64_t n, double* out, cudaStream_t s);
// a, b out of the interleaved fill buffer into planar arrays.
cudaError_t launch_unpack_ab(const float4* isab, float* a, float* b, int64_t n, cudaStream_t s);
int fill_words(int nx, int ny, int nz);
int fill_front_blocks(int nx, int ny, int nz);
cudaError_t launch_fill_pack(const int* stamp, unsigned* k, int nx, int ny, int nz, cudaStream_t s);
struct ForceArgs {
  const float* d;       // I'_s - m
  const float* m;
  const float* r;
  float* u;             // r + dr
  float* partials;      // per CTA: sum |dr|, sum |r|
  int norm_lo, norm_hi; // only planes [norm_lo, norm_hi) enter those sums (all if norm_hi <= norm_lo)
  const int* stop;
  int nx, ny, nz;
  int force_mode;
  int u_is_dr;          // write u = dr instead of r + dr
};
int force_blocks(int64_t n, int max_parts);
cudaError_t launch_force_dm(const ForceArgs& f, int blocks, cudaStream_t s);
// Lower and upper median of the non-negative entries of a (radix select).
// work: median_work_words() unsigned words; results: work[65536] = count,
// work[65537 + 3] = lower median bits, work[65537 + 7] = upper median bits.
size_t median_work_words();
cudaError_t launch_median(const float* a, int64_t n, unsigned* work, cudaStream_t s);
// *out = mean of the two medians in work (double), -1 when there are none.
cudaError_t launch_median_finish(const unsigned* work, double* out, cudaStream_t s);
// *out = voxels the fill left unfilled, from its counters.
cudaError_t launch_fill_remaining(const int* cnt, int passes, int* out, cudaStream_t s);
// out = a + b elementwise.
cudaError_t launch_add(const float* a, const float* b, float* out, int64_t n, cudaStream_t s);

// ----------------------------------------------------------------------------
// Evaluation metrics, metrics.cu (Sec. 2.4.3)
// ----------------------------------------------------------------------------
cudaError_t metric_nmi(const float* a, const float* b, int64_t n, int bins, double* out, cudaStream_t s);
// synchronises s (the hysteresis passes run until nothing changes)
cudaError_t metric_canny(const float* img, uint8_t* edges, int nx, int ny, int nz, float sigma, float t_low,
                         float t_high, cudaStream_t s);
cudaError_t metric_edge_rmse(const uint8_t* a, const uint8_t* b, int64_t n, double* out, cudaStream_t s);

// ----------------------------------------------------------------------------
// Small kernels, misc.cu
// ----------------------------------------------------------------------------
cudaError_t launch_max_abs(const float* v, int64_t n, float* out, cudaStream_t s);
// Sums of two arrays into per-CTA double partials, then the shift Is_out = Is + delta.
cudaError_t launch_global_shift(const float* Im, const float* Is, float* Is_out, int64_t n,
                                double* scratch /* >= 2*kShiftBlocks+1 doubles */,
                                float* delta_out, cudaStream_t s);
constexpr int kShiftBlocks = 592;
cudaError_t launch_down2(const float* in, float* out, int nx, int ny, int nz, cudaStream_t s);
cudaError_t launch_up2(const float* rc, float* rf, int nx, int ny, int nz, cudaStream_t s);
// Reduce per-CTA partial norms to l^(k), append to the level history, update the stop flag.
struct NormState {
  float* hist;          // [cap] l values of the current level
  double* sums;         // [cap][2] sum |dr|, sum |r| behind each l
  int* iter;            // iterations run at the current level
  int* stop;            // stop flag
  int cap;
  int window;
  float eps;
  // in-graph loop (conditional WHILE node): iterations left in this launch; the
  // kernel decrements it and sets the loop condition to (left > 0 and not stopped)
  int* budget;
  cudaGraphConditionalHandle cond;
  int use_cond;
};
// *p = v (a one-thread kernel, stream-ordered)
cudaError_t launch_set_int(int* p, int v, cudaStream_t s);

// Programmatic dependent launch of the per-iteration kernels (box pass, the two
// Gaussian passes, the norm): a kernel launched this way may be scheduled while
// its predecessor on the stream finishes; it calls pdl_wait() before touching
// global memory, which returns once every prerequisite grid has completed and
// its writes are visible, and pdl_release() to let its own successor be
// scheduled once all of its CTAs run.  Both are no-ops for a normal launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}
// Raise the release threshold of the current device's default memory pool (once
// per device), so that the scratch the kernel-level calls allocate stream-ordered
// is reused from call to call instead of being unmapped at each synchronisation.
void keep_pool_memory();
cudaError_t launch_norm_finalize(const float* partials, int nparts, NormState st, cudaStream_t s);
// One block per volume: NormState and partials of volume p in the tables.
struct NormBatch {
  int count;
  const float* partials[kMaxBatch];
  int nparts[kMaxBatch];
  NormState st[kMaxBatch];
};
cudaError_t launch_norm_finalize_batch(const NormBatch& nb, int count, cudaStream_t s);
// Warp of many volumes in one launch (warp.cu); args: Im, r, m, dims per volume.
struct WarpBatch {
  int count;
  int offset[kMaxBatch + 1];
  const float* Im[kMaxBatch];
  const float* r[kMaxBatch];
  float* m[kMaxBatch];
  int nx[kMaxBatch], ny[kMaxBatch], nz[kMaxBatch];
  const int* stop[kMaxBatch];
};
cudaError_t launch_warp_batch(const WarpBatch& wb, int total_blocks, cudaStream_t s);
constexpr int kWarpBatchThreads = 128;
// The z-marching warp over a work table whose offsets count warp_z_blocks of
// each pair's volume (warp.cu).
int warp_z_blocks(int nx, int ny, int nz);
cudaError_t launch_warp_z_batch(const WarpBatch& wb, int total_blocks, cudaStream_t s);
// Deterministic fixed-order sum of per-CTA float partials (stride 2, component c) into *out.
cudaError_t launch_partials_sum(const float* partials, int nparts, int comp, double* out,
                                cudaStream_t s);

}  // namespace disc
