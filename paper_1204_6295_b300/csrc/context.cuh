// The registration context (disc_ctx) and its per-level state, shared by the
// single-pair API (api.cu) and the batched API (batch.cu).
#pragma once

#include <nvtx3/nvToolsExt.h>

#include "internal.cuh"

namespace disc {

// NVTX range for the profilers' timelines (header-only NVTX 3: a no-op unless a
// tool is attached).  The library marks its calls, each level's iterations and,
// when kernels are launched one by one (no graph replay), each pass.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};


struct Level {
  int nx = 0, ny = 0, nz = 0;
  size_t N = 0;
  float* Im = nullptr;   // moving image (CT) at this level
  float* Is = nullptr;   // static image (CBCT, shifted) at this level
  float* zs = nullptr;   // (I_s - E(S)) / STD(S) over the patch
  float* m = nullptr;    // warped CT I_m(x + r(x))
  float* r = nullptr;    // field [3][N]
  float* u = nullptr;    // r + dr [3][N]
  float* t = nullptr;    // z-filtered field [3][N] (Gaussian scratch)
  float* hist = nullptr; // l^(k) history
  double* hsum = nullptr;   // [hist_cap][2] sum |dr|, sum |r| behind each l^(k)
  int hist_cap = 0;
  int norm_lo = 0, norm_hi = 0;   // planes entering those sums (all when norm_hi <= norm_lo)
  // mask and fill (mask_mode 1)
  float* sd = nullptr;   // STD(S)
  float* ab = nullptr;   // a [N] then b [N] (the ratio a of the median a_m)
  float4* isab = nullptr;   // [N] (I_s, a, b, 0): the mask pass writes it, the fill completes it
  float* dm = nullptr;   // I'_s - m of the masked correction
  int* stamp = nullptr;  // 0 known, p filled by pass p, -1 not filled
  unsigned* kbits = nullptr;   // [2][fill_words] known-voxel bit masks of the fill passes
  int* flist = nullptr;        // [N] a fill pass's front; then [fill_front_blocks + 1] block offsets, length
  int* cnt = nullptr;    // [fill_passes + 2] masked voxels, voxels filled per pass; then the pass counter
  BoxPlan pa{};          // iteration pass of this context (possibly the wide-tile one)
  BoxPlan pn{};          // iteration pass on the 32 x 16 tiling (the batched launches)
  BoxPlan pm{};          // kModeMaskAB
  GaussPlan pb{};
  cudaGraphExec_t graph = nullptr;   // n iterations unrolled (graph_iters = n)
  int graph_iters = 0;
  long long graph_kernels = 0;       // kernel nodes of `graph`
  cudaGraphExec_t loop = nullptr;    // one iteration inside a conditional WHILE node
  long long loop_kernels = 0;        // kernel nodes of one iteration of `loop`
  bool sep_warp = false;             // this level's warp runs in its own kernel
};


}  // namespace disc

struct disc_ctx {
  disc_params p{};
  int device = 0;
  int num_sms = disc::kNumSMs;
  cudaStream_t user = nullptr;
  cudaStream_t s = nullptr;
  cudaStream_t side = nullptr;   // captures the bodies of the fill loops
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  int hx = 0, hy = 0, hz = 0, R = 0;
  float w[2 * DISC_MAX_GAUSS_RADIUS + 1] = {};
  int nx = 0, ny = 0, nz = 0;
  int L = 0;
  bool have_images = false;
  disc::Level lev[DISC_MAX_LEVELS];
  float qs_m = 1.0f, qs_s = 1.0f;
  float* partials = nullptr;
  int max_parts = 0;
  int* d_iter = nullptr;     // [DISC_MAX_LEVELS]
  int* d_stop = nullptr;     // [DISC_MAX_LEVELS]
  int* d_err = nullptr;      // device error word of the box kernels (d_stop + DISC_MAX_LEVELS)
  int* d_budget = nullptr;   // [DISC_MAX_LEVELS] iterations left in the running loop graph
  double* d_scratch = nullptr;
  float* d_maxabs = nullptr; // [2]
  float mask_hu0 = 0.0f, mask_am = 0.0f;   // Eq. 7 thresholds (mask_mode 1)
  unsigned* d_mwork = nullptr;              // median work words
  int cur_level = 0;
  int cur_iter = 0;
  disc_status sticky = DISC_OK;
  bool use_graphs = true;
  bool use_loop = true;      // conditional-node loop graphs (with a stop rule; else unrolled graphs)
  long long launches = 0;    // kernels disc_iterate has launched (disc_get_launch_count); -1: not kept
  // where the next iteration's warp runs: 1 in a kernel of its own after the
  // Gaussian, 0 (the default) inside the Gaussian's last pass, the xy pass,
  // which holds r in registers and gathers I_m tile by tile
  int separate_warp = 0;
};


namespace disc {
// Helpers of api.cu used by the batched API.
// Zero level l's iteration counter and stop flag, in stream order on s (the
// batch's stream, where the batched kernels that use them run).
cudaError_t ctx_reset_level_counters(disc_ctx* c, int l, cudaStream_t s);
// Grow the context's per-CTA norm partials to at least n (float2 each); drops
// its own captured graphs, which hold the old buffer.
cudaError_t ctx_reserve_partials(disc_ctx* c, int n);
BoxArgs ctx_box_args(const disc_ctx* c, int l);       // iteration-mode box arguments of level l
GaussArgs ctx_gauss_args(const disc_ctx* c, int l);   // Gaussian arguments of level l (with warp)
NormState ctx_norm_state(const disc_ctx* c, int l);
// Queue up to `budget` iterations of the schedule on c->s from the current
// level and iteration, up-sampling each level finished on the way (Algorithm
// A1).  touched/ntouched: the levels that ran iterations (may be NULL);
// queued: the number of iterations queued (may be NULL).  No stream
// ordering with the caller's stream: the caller provides it.
cudaError_t ctx_advance(disc_ctx* c, long long budget, int* touched, int* ntouched, long long* queued);
}  // namespace disc
