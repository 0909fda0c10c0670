/*
 * disc.h -- C ABI of the B300 (sm_103a) DISC library, libdisc.so.
 *
 * DISC ("Deformation with Intensity Simultaneously Corrected", Zhen et al.,
 * arXiv 1204.6295) registers a planning CT (the moving image I_m) to a CBCT
 * (the static image I_s) with demons, correcting the CBCT intensity at every
 * iteration by matching the first two moments of a patch around each voxel
 * to the same patch of the deformed CT.
 *
 * Problem statement (Sec. 2.1, Sec. 2.2): given I_m and I_s on one grid,
 * find a displacement field r with I_m(x + r(x)) = I_s(x), together with the
 * corrected CBCT I'_s = a I_s + b (Eqs. 2-6).  Algorithm A1 gives the
 * procedure this library runs: a global intensity shift, a multi-resolution
 * pyramid, then per level and per iteration: warp, moment matching,
 * correction, demons force (Eq. 1), field update and Gaussian regularisation.
 *
 * Conventions shared by every call
 *  - Layout: images are float32 [nz][ny][nx] (x fastest, C order).  Fields
 *    are float32 structure-of-arrays [3][nz][ny][nx], components (x, y, z),
 *    in voxel units of the grid they are defined on.
 *  - Memory kinds: DISC_MEM_HOST pointers are ordinary host memory (pinned
 *    or pageable); DISC_MEM_DEVICE pointers are device memory on the
 *    context's device.  The library never keeps a caller pointer after a
 *    call returns, and the caller owns every buffer it passes.
 *  - Streams: every call is ordered on the caller's stream given at
 *    creation (a cudaStream_t; NULL = the legacy default stream): the work
 *    runs on a library stream that waits for the caller's stream on entry and
 *    that the caller's stream waits for on exit (CUDA events), so that the
 *    library can replay CUDA graphs.  Calls that write host memory
 *    synchronise before returning.
 *  - Errors: every call returns a disc_status by value; no C++ exception
 *    crosses this boundary.  The first CUDA error seen by a context is
 *    sticky: later calls on it return DISC_ERR_STATE until disc_destroy.
 *  - Threads: a context is not thread-safe; distinct contexts are independent.
 *  - Kernel-level calls (disc_k_*) take device pointers only, enqueue on the
 *    given stream and return without synchronising.
 */
#ifndef DISC_H
#define DISC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct disc_ctx disc_ctx;       /* opaque, owned by the library */

typedef enum {
  DISC_OK = 0,
  DISC_ERR_ARG = 1,      /* NULL pointer, bad enum or parameter value      */
  DISC_ERR_SHAPE = 2,    /* sizes inconsistent or outside supported range  */
  DISC_ERR_STATE = 3,    /* call out of order, or context already failed   */
  DISC_ERR_OOM = 4,      /* device allocation failed                        */
  DISC_ERR_CUDA = 5,     /* a CUDA runtime call failed                      */
  DISC_ERR_TIMEOUT = 6   /* a bounded device-side wait gave up              */
} disc_status;

enum { DISC_MEM_HOST = 0, DISC_MEM_DEVICE = 1 };

/* Demons force, Eq. (1).  THIRION is the first (passive) term alone; DOUBLE
 * is the double-force form Eq. (1) prints.  The image difference is taken
 * as (I'_s - I_m^(k)) so that adding dr moves I_m(x + r) toward I_s under
 * the Sec. 2.1 convention I_m(x + v(x)) = I_s(x). */
enum { DISC_FORCE_THIRION = 0, DISC_FORCE_DOUBLE = 1 };

#define DISC_MAX_LEVELS 8
#define DISC_MAX_HALF_PATCH 15   /* patch sizes up to 31 voxels per axis   */
#define DISC_MAX_GAUSS_RADIUS 16

typedef struct {
  int32_t patch[3];      /* odd patch sizes (px, py, pz); Sec. 3.3 uses 3x3x3 */
  float gauss_sigma;     /* Gaussian sigma of the field regularisation, voxels */
  int32_t gauss_radius;  /* taps |i| <= radius; 0 = ceil(3 sigma)              */
  int32_t levels;        /* pyramid levels, >= 1 (Sec. 2.3 uses 2)             */
  int32_t iters[DISC_MAX_LEVELS];  /* iterations per level, coarsest first     */
  float stop_eps;        /* Sec. 2.3 stop rule threshold (1e-4); <= 0 = fixed counts */
  int32_t stop_window;   /* Sec. 2.3 compares l^(k-10) with l^(k): 10          */
  int32_t force_mode;    /* DISC_FORCE_THIRION or DISC_FORCE_DOUBLE            */
  int32_t global_shift;  /* 1 = shift I_s by mean(I_m) - mean(I_s) (Sec. 2.3)  */
  float var_floor;       /* patch variance (HU^2) at or below which STD = 0    */
  /* Mask and fill of a, b (Eqs. 7-10, Algorithm A1 step 2).  With mask_mode 1
   * every iteration sets xi = 1 where |I_m^(k) - I_s| > HU0, where a is outside
   * [a_min, a_max] or undefined (STD(S) = 0), and replaces a, b there by the
   * weighted mean of Eqs. 8-10 over the known voxels of the box T, in Jacobi
   * passes (a pass uses the voxels known before it) until none is left, a pass
   * fills nothing, or fill_passes passes have run; a voxel never filled keeps
   * a = b = 0.  HU0 = hu0_factor |dHU| (dHU the global shift, computed even
   * when it is not applied); a_min = a_lo a_m, a_max = a_hi a_m with a_m the
   * median of STD(M)/STD(S) at the finest level with r = 0, fixed at
   * disc_set_images.  Weights exp(-min((I_s(i) - I_s(x))^2 / h^2, 80)). */
  int32_t mask_mode;     /* 0: off (xi = 0 everywhere); 1: on                  */
  float hu0_factor;      /* Sec. 2.3: 2                                         */
  float a_lo, a_hi;      /* Sec. 2.3: 0.5, 1.5                                  */
  float fill_h;          /* h of Eq. 10, HU (the paper gives none): 50          */
  int32_t fill_t[3];     /* odd box T sizes (x, y, z), Sec. 2.3: 7, 7, 3         */
  int32_t fill_passes;   /* at most this many fill passes per iteration: 32     */
  /* What the Gaussian regularises: 0 = the total field, r <- G * (r + dr)
   * (Algorithm A1 steps 5-6); 1 = the increment, r <- r + G * dr (the order of
   * Sec. 2.1: smooth dr, then add it to the field). */
  int32_t smooth_mode;
  /* Bounds of |I_m| and |I_s| (after the global shift) from which the
   * fixed-point scales of the patch sums are derived (disc_qscale); 0 = the
   * images' own largest magnitudes.  A z slab of a larger volume passes the
   * whole volume's maxima so that its sums and moments are those of the whole
   * volume bit for bit.  A bound below the images' own maximum is rejected
   * by disc_set_images (DISC_ERR_ARG): the sums could overflow. */
  float quant_max[2];
  /* Finest-level z planes [lo, hi) whose voxels enter the sums of l^(k)
   * (Sec. 2.3), halved (rounding up) at each coarser level; 0 0 = every
   * plane.  A z slab of a larger volume counts its interior only, so that the
   * slabs' sums add up to the whole volume's (disc_get_norm_sums). */
  int32_t norm_planes[2];
} disc_params;

/* Fill *p with defaults: patch 3x3x3, sigma 1, radius 0, 2 levels of 50
 * iterations, stop_eps 0 (fixed counts), window 10, THIRION, global shift on,
 * var_floor 1e-6, mask off (hu0_factor 2, a_lo 0.5, a_hi 1.5, fill_h 50,
 * fill_t 7x7x3, fill_passes 32), smooth_mode 0, quant_max 0 0, norm_planes
 * 0 0.  Returns
 * DISC_ERR_ARG for NULL. */
disc_status disc_params_default(disc_params* p);

/* Human-readable name of a status code (static storage, never NULL). */
const char* disc_status_str(disc_status s);

/* Create a context on CUDA device `device`, ordered on `cuda_stream`
 * (a cudaStream_t, or NULL for the legacy default stream).  Validates *p:
 * odd patch sizes in [1, 31], sigma > 0, levels in [1, 8], iters >= 0.
 * On success *out owns device resources until disc_destroy. */
disc_status disc_create(const disc_params* p, int device, void* cuda_stream,
                        disc_ctx** out);

/* Load the CT (moving, I_m) and CBCT (static, I_s) images, both
 * [nz][ny][nx] float32, from host or device memory (mem_kind).  Applies the
 * global shift (Sec. 2.3, Algorithm A1 first line), builds the pyramid by
 * 2x2x2 averaging (ceil(n/2) voxels per axis per level), precomputes each
 * level's CBCT patch statistics, and sets r = 0 at the coarsest level
 * (Algorithm A1).  Sizes: every axis >= 1.  Replaces any previous images. */
disc_status disc_set_images(disc_ctx* ctx, const float* ct_moving,
                            const float* cbct_static, int32_t nx, int32_t ny,
                            int32_t nz, int mem_kind);

/* Advance the schedule of Algorithm A1 by at most `max_iters` iterations
 * (-1 = run to the end of the schedule), coarsest level first, up-sampling
 * r to the next level at each level's end.  One iteration = warp, patch
 * moments of I_m^(k) and I_s, correction I'_s = a I_s + b (Eqs. 5-6),
 * Thirion or double force (Eq. 1), r += dr, r <- G_sigma * r.  With
 * stop_eps > 0 a level ends early once l^(k-window) - l^(k) <= stop_eps,
 * l^(k) = sum|dr^(k+1)| / sum|r^(k)| (Sec. 2.3).
 * If iters_done or last_l is non-NULL the call synchronises the stream and
 * returns the iterations executed by this call and the last l^(k) (+inf
 * while sum|r| = 0); otherwise it returns without synchronising. */
disc_status disc_iterate(disc_ctx* ctx, int32_t max_iters, int32_t* iters_done,
                         float* last_l);

/* Copy the displacement field on the finest grid, [3][nz][ny][nx] float32,
 * in finest-grid voxel units, to `out` (host or device).  Before the
 * schedule reaches the finest level, the current field is up-sampled
 * through the remaining levels first. */
disc_status disc_get_field(disc_ctx* ctx, float* out, int mem_kind);

/* Copy the field r of pyramid level `level` (0 = finest) as the context holds
 * it: [3][nz][ny][nx] of that level's grid, in that level's voxel units (the
 * layout disc_set_field takes).  No up-sampling; host or device `out`.
 * DISC_ERR_ARG for a level outside [0, levels). */
disc_status disc_get_level_field(disc_ctx* ctx, int32_t level, float* out, int mem_kind);

/* Copy the corrected CBCT I'_s (Sec. 2.2, last paragraph), computed from
 * the current field at the current level, [nz][ny][nx] of that level. */
disc_status disc_get_corrected(disc_ctx* ctx, float* out, int mem_kind);

/* Replace the field of pyramid level `level` (0 = finest) with `r`
 * ([3][nz][ny][nx] of that level) and make it the current level with its
 * iteration count reset: resuming from a saved field. */
disc_status disc_set_field(disc_ctx* ctx, int32_t level, const float* r,
                           int mem_kind);

/* Differentiable form on the context's own data (not in the paper): for a
 * field r on pyramid level `level` ([3][nz][ny][nx] of that level, its voxel
 * units), the SSD between the warped CT and the moment-matched CBCT of that
 * level, L(r) = sum_x (I_m(x + r(x)) - I'_s(x))^2 (as disc_k_ssd_loss, with the
 * context's CBCT normalisation zs and fixed-point scale), into *loss (host
 * double, may be NULL), and dL/dr into grad (same layout and memory kind as r,
 * may be NULL; as disc_k_ssd_grad: cubic patches of half size 1..8 only, else
 * DISC_ERR_SHAPE).  At least one of loss and grad is required.  Does not change
 * the registration's state (field, level, iteration count); the next
 * disc_iterate rebuilds the scratch this call uses.  Synchronises when loss is
 * requested or the buffers are host memory. */
disc_status disc_ssd(disc_ctx* ctx, int32_t level, const float* r, double* loss, float* grad, int mem_kind);

/* Position in the schedule: current level (0 = finest) and iterations
 * already run at it.  *dims receives that level's (nx, ny, nz) if non-NULL. */
disc_status disc_get_progress(disc_ctx* ctx, int32_t* level, int32_t* iter,
                              int32_t dims[3]);

/* Kernel launches disc_iterate has issued on this context since its creation
 * (the paper has no counterpart; evidence that the hot path ran as kernels):
 * each replay of a level's iteration graph adds the graph's kernel nodes, each
 * up-sampling between levels adds one.  Exact with fixed iteration counts and
 * the mask off.  With the stop rule, a level's iteration loop runs a number of
 * times decided on the device: its body's kernels are counted once per
 * iteration the call allows.  The mask's fill passes (a conditional loop
 * inside each iteration) are not counted.  -1 after a call that ran without
 * graphs (DISC_SW_NO_GRAPH), whose launches are not counted.  Host memory. */
disc_status disc_get_launch_count(disc_ctx* ctx, int64_t* launches);

/* Copy the l^(k) history of `level` (up to `cap` values, one per iteration
 * run there) into host memory; *count receives the number written. */
disc_status disc_get_norm_history(disc_ctx* ctx, int32_t level, float* out,
                                  int32_t cap, int32_t* count);

/* The two sums behind each l^(k) of `level`, sum_x |dr(x)| and sum_x |r(x)|
 * over the planes of norm_planes, as doubles: out[2k], out[2k + 1] for each
 * iteration k run there (up to `cap` iterations), *count receives the number
 * of iterations written.  Host memory. */
disc_status disc_get_norm_sums(disc_ctx* ctx, int32_t level, double* out, int32_t cap, int32_t* count);

/* The convergence norm and stop rule of Sec. 2.3 for sums gathered outside a
 * context, e.g. a z-slab split of one volume over several ranks, where each
 * rank's interior sums (disc_get_norm_sums with norm_planes set) are added over
 * the ranks.  sums[2k] = sum |dr|, sums[2k + 1] = sum |r| of iterations
 * k = 0 .. count - 1 of one level (host memory).  l_out (host, may be NULL)
 * receives l^(k) = sum |dr| / sum |r| for every k (float; +inf while sum |r| = 0);
 * *stop is 1 when the rule ends the level after its last iteration:
 * count - 1 >= window, both l^(count - 1 - window) and l^(count - 1) finite, and
 * their difference <= eps (eps <= 0: never).  The same arithmetic as a
 * context's own norm kernel.  No device work: callable without a GPU. */
disc_status disc_norm_stop_rule(const double* sums, int32_t count, int32_t window, float eps,
                                float* l_out, int32_t* stop);

/* The mask thresholds fixed by disc_set_images (mask_mode 1): HU0 and a_m
 * (a_min = a_lo a_m, a_max = a_hi a_m).  DISC_ERR_STATE before images or
 * with the mask off.  Any pointer may be NULL. */
disc_status disc_get_mask_constants(disc_ctx* ctx, float* hu0, float* a_m);

/* Sec. 2.4.3 metrics of the registration at its current level: NMI (bins)
 * and the Canny edge RMSE of Eq. 11 (sigma, t_low, t_high; see
 * disc_k_canny) between the warped CT I_m(x + r(x)) and the corrected CBCT
 * I'_s.  Host outputs (either may be NULL); synchronises. */
disc_status disc_get_metrics(disc_ctx* ctx, int32_t bins, float sigma, float t_low, float t_high,
                             double* nmi, double* rmse_edge);

/* The averages of the correction coefficients (Sec. 3.4 shows their maps and
 * their averages over the iterations): for the current field at the current
 * level, a = STD(M)/STD(S) and b = E(M) - a E(S) of Eqs. 5-6 (with the mask on,
 * after the mask and fill of Eqs. 7-10, as the next iteration would use them),
 * averaged over the voxels where they are defined (STD(S) > 0; with the mask,
 * the voxels known or filled).  Host outputs (any may be NULL; not all); NaN
 * means when no voxel qualifies.  Synchronises; the registration's state is
 * unchanged.  A caller logs the averages per iteration by iterating one step
 * at a time. */
disc_status disc_get_correction_means(disc_ctx* ctx, double* mean_a, double* mean_b, int64_t* count);

/* Release every resource of the context.  NULL is accepted. */
disc_status disc_destroy(disc_ctx* ctx);

/* ---------------------------------------------------------------------
 * Batched registration: many CT/CBCT pairs of uneven size advanced together
 * (the workloads' batched form; not in the paper).  Each pair runs exactly the
 * single-pair computation (bit-identical fields), but one iteration of all
 * pairs is one launch per step of the iteration over a work table of every
 * pair's tiles, a level's iterations are one CUDA graph, and the tile
 * scheduling of the moment/force launch is tuned per level at first use.
 * All pairs share the parameters and the schedule.  Cubic patches of 3..15
 * voxels and Gaussian radius 1..8 only (DISC_ERR_ARG otherwise).
 * With mask_mode 1 (Eqs. 7-10) the number of fill passes differs per pair and
 * iteration, so the pairs run their own single-pair schedules concurrently on
 * their own streams, forked from and joined to the batch's stream in each
 * disc_batch_iterate call (bit-identical to separate runs as well); the tuning
 * getters then return DISC_ERR_STATE.
 * ------------------------------------------------------------------- */
typedef struct disc_batch disc_batch;

/* Create a batch of npairs (1..64) pairs on `device`, ordered on `cuda_stream`. */
disc_status disc_batch_create(const disc_params* p, int device, void* cuda_stream,
                              int32_t npairs, disc_batch** out);

/* Load pair `pair`'s images (as disc_set_images).  Allowed only before the
 * batch has iterated (or after disc_batch_restart); DISC_ERR_STATE otherwise. */
disc_status disc_batch_set_images(disc_batch* b, int32_t pair, const float* ct_moving,
                                  const float* cbct_static, int32_t nx, int32_t ny,
                                  int32_t nz, int mem_kind);

/* Reset every pair's field to 0 at the coarsest level and the schedule to its
 * start (images and patch statistics are kept). */
disc_status disc_batch_restart(disc_batch* b);

/* Advance the shared schedule by at most max_iters iterations (-1 = to the
 * end), as disc_iterate does for one pair; *iters_done (may be NULL)
 * receives the iterations run.  Does not synchronise, except at the first
 * iteration of a level, where the tuning launches are timed. */
disc_status disc_batch_iterate(disc_batch* b, int32_t max_iters, int32_t* iters_done);

/* Copy pair `pair`'s field on its finest grid (as disc_get_field). */
disc_status disc_batch_get_field(disc_batch* b, int32_t pair, float* out, int mem_kind);

/* Tuning chosen for `level`: work items of the moment/force launch, its grid
 * (equal to items, or one wave of persistent CTAs), and the z chunking: a
 * positive value k lengthens each pair's single-pair chunk k times, a
 * negative value -c sets chunks of c planes (capped at each pair's depth), 0
 * the wide-tile kernel (items = the (tile, plane) pairs of all pairs, capped
 * at 2^30).  DISC_ERR_STATE before the level has run. */
disc_status disc_batch_get_tuning(disc_batch* b, int32_t level, int32_t* items, int32_t* grid,
                                  int32_t* zmult);

/* Which moment/force kernel `level` runs: *tma = 2 for the wide-tile kernel
 * (32 x 32 tiles, the (tile, plane) pairs of all pairs shared evenly by one
 * wave of CTAs), 1 for the bulk-tensor-copy-fed kernel on 32 x 16 tiles, 0 for
 * the per-thread-load kernel on 32 x 16 tiles.  Both bulk-copy kernels need
 * every pair's level to meet their conditions (nx a multiple of 4, extents of
 * at least one staging box, 16-byte aligned buffers); the tuner times the wide
 * kernel against the 32 x 16 tilings and keeps the fastest.  DISC_ERR_STATE
 * before the level has run. */
disc_status disc_batch_get_box_path(disc_batch* b, int32_t level, int32_t* tma);

/* Tuning of `level`'s Gaussian and warp (Algorithm A1 step 6 and the warp of
 * step 1 for the next iteration): *zlen = the z chunk length of the Gaussian's
 * z pass, its first (0: each pair's single-pair plan; else chunks of that many
 * planes, capped at each pair's depth) and *separate_warp = 1 when the warp
 * runs as the z-marching warp kernel after the Gaussian, 0 when it runs inside
 * its last pass, the xy pass.  At the level's first iteration the tuner times
 * the z and xy passes (and the warp) on scratch copies of r and m for chunks
 * of the pairs' plans, 16, 32
 * and 64 planes, with either placement, and keeps the default (fused, the
 * plans) unless a choice is at least 2% faster.  Bitwise neutral: every output
 * is the same sum in the same order either way.  Either output may be NULL.
 * DISC_ERR_STATE before the level has run (and always with mask_mode 1). */
disc_status disc_batch_get_gauss_tuning(disc_batch* b, int32_t level, int32_t* zlen,
                                        int32_t* separate_warp);

/* Pin the tuning of `level` instead of letting the autotuner time it.  zmult
 * non-zero: the 32 x 16 tilings with z chunking `zmult` (as
 * disc_batch_get_tuning reports it) and the moment/force launch's grid: 0 for
 * one CTA per work item, g > 0 for min(g, items) persistent CTAs striding over
 * the work table.  zmult 0: the wide-tile kernel with one wave of CTAs (grid
 * 0) or g CTAs sharing the planes (DISC_ERR_CUDA at the level's first
 * iteration when a pair's level cannot take it).  Takes effect at the level's
 * next iteration (the level's graph is rebuilt); synchronises the batch's
 * stream.  The fields do not depend on the tuning (bit for bit). */
disc_status disc_batch_pin_tuning(disc_batch* b, int32_t level, int32_t zmult, int32_t grid);

/* Release the batch and every pair context.  NULL is accepted. */
disc_status disc_batch_destroy(disc_batch* b);

/* ---------------------------------------------------------------------
 * Kernel-level calls: one hot-path step on caller-owned device buffers.
 * All pointers are device pointers on the current device; work goes on
 * `stream` (cudaStream_t, NULL = legacy default stream).  `patch` is the
 * odd patch size per axis; `qscale` is the fixed-point scale (a power of
 * two, see disc_qscale).  Buffers may not overlap unless stated.  Calls that
 * need scratch take it stream-ordered from the device's default memory pool
 * and raise that pool's release threshold, so that repeated calls reuse it.
 * ------------------------------------------------------------------- */

/* Fixed-point scale 2^e used for exact integer patch sums of an image
 * whose largest magnitude is `max_abs`, for patches of `patch` voxels:
 * the largest e with |q| = |v| 2^e small enough that every patch sum of q^2
 * fits in 63 bits.  Returns 0 for invalid arguments. */
float disc_qscale(float max_abs, const int32_t patch[3]);

/* Largest |v| over n floats, written to *out (device float). */
disc_status disc_k_max_abs(const float* v, int64_t n, float* out, void* stream);

/* Global intensity shift (Sec. 2.3): Is_out = Is + (mean(Im) - mean(Is)),
 * means over n voxels; *delta_out (device float, may be NULL) gets the
 * shift.  Is_out may equal Is. */
disc_status disc_k_global_shift(const float* Im, const float* Is, float* Is_out,
                                int64_t n, float* delta_out, void* stream);

/* 2x2x2 mean down-sampling (pyramid build, Sec. 2.3): in [nz][ny][nx] ->
 * out [ceil(nz/2)][ceil(ny/2)][ceil(nx/2)]; a partial cell averages the
 * voxels it has. */
disc_status disc_k_downsample2(const float* in, float* out, int32_t nx, int32_t ny,
                               int32_t nz, void* stream);

/* Field up-sampling to the next finer level (Algorithm A1): fine voxel i
 * samples the coarse field at (i - 0.5)/2 per axis (clamped), trilinear,
 * times 2.  rc [3][cz][cy][cx] -> rf [3][nz][ny][nx], where cz = ceil(nz/2)
 * and likewise for y and x. */
disc_status disc_k_upsample_field2(const float* rc, float* rf, int32_t nx,
                                   int32_t ny, int32_t nz, void* stream);

/* CBCT patch normalisation for Eqs. (5)-(6): zs = (I_s - E(S)) / STD(S)
 * over the truncated patch around each voxel (0 where Var(S) <= var_floor).
 * Then I'_s = zs * STD(M) + E(M) equals a I_s + b. */
disc_status disc_k_static_norm(const float* Is, float* zs, int32_t nx, int32_t ny,
                               int32_t nz, const int32_t patch[3], float qscale,
                               float var_floor, void* stream);

/* Trilinear warp (Sec. 2.1; Sec. 2.3 kernel 5): m(x) = I_m(x + r(x)), the
 * sample position clamped to the volume per axis.  Im, m [nz][ny][nx];
 * r [3][nz][ny][nx].  ny, nz <= 65535.  m must not alias Im or r. */
disc_status disc_k_warp(const float* Im, const float* r, float* m, int32_t nx,
                        int32_t ny, int32_t nz, void* stream);

/* One iteration front (Algorithm A1 steps 1, 3, 4, 5):
 * m = I_m(x + r(x)); E(M), STD(M) over the truncated patch (Eq. 3);
 * I'_s = zs STD(M) + E(M) (= a I_s + b of Eqs. 5-6); dr from Eq. (1) with
 * I'_s in place of I_s; u = r + dr.
 * Optional outputs (NULL to skip): m_out receives m; d_out receives
 * I'_s - m (the corrected CBCT relative to the warped CT, the quantity the
 * force is computed from).  norms_out (device double[2], may be NULL)
 * receives sum|dr| and sum|r|.  u must not alias r.  Temporary device
 * memory is taken from the stream-ordered allocator. */
disc_status disc_k_pass_a(const float* Im, const float* zs, const float* r, float* u,
                          float* m_out, float* d_out, double* norms_out,
                          int32_t nx, int32_t ny, int32_t nz, const int32_t patch[3],
                          float qscale, float var_floor, int32_t force_mode,
                          void* stream);

/* The moment, correction, force and update pass of disc_k_pass_a on a warped
 * image m (= I_m(x + r(x)), e.g. from disc_k_warp) given by the caller
 * (Eqs. 3-6, Eq. 1, Algorithm A1 steps 1, 3, 4, 5).  Same outputs as
 * disc_k_pass_a except m. */
disc_status disc_k_force_update(const float* m, const float* zs, const float* r, float* u,
                                float* d_out, double* norms_out, int32_t nx, int32_t ny,
                                int32_t nz, const int32_t patch[3], float qscale,
                                float var_floor, int32_t force_mode, void* stream);

/* Differentiable form (not in the paper): the SSD between the warped CT and
 * the moment-matched CBCT, L(r) = sum_x (I_m(x + r(x)) - I'_s(x))^2 with
 * I'_s = zs STD(M) + E(M) over the truncated patch (Eqs. 3-6; the CBCT side zs
 * is fixed).  *loss_out (device double) receives L.  Temporary device memory
 * comes from the stream-ordered allocator. */
disc_status disc_k_ssd_loss(const float* Im, const float* zs, const float* r,
                            double* loss_out, int32_t nx, int32_t ny, int32_t nz,
                            const int32_t patch[3], float qscale, float var_floor,
                            void* stream);

/* Gradient dL/dr of the loss above, [3][nz][ny][nx], by adjoint kernels:
 * the patch statistics are recomputed (not stored), the adjoint of the
 * moment matching is a truncated box sum of three per-voxel coefficients,
 * and the warp's adjoint is the analytic trilinear derivative (zero along an
 * axis whose sample position is clamped).  Cubic patches only (half size 1..8;
 * other patches return DISC_ERR_SHAPE).  loss_out (may be NULL) also receives
 * L, summed in the same pass from the same d = I'_s - m (its float partial
 * sums are grouped by that pass's CTAs, so it can differ from
 * disc_k_ssd_loss's value in the last bits).  grad must not alias r. */
disc_status disc_k_ssd_grad(const float* Im, const float* zs, const float* r, float* grad,
                            double* loss_out, int32_t nx, int32_t ny, int32_t nz,
                            const int32_t patch[3], float qscale, float var_floor,
                            void* stream);

/* Allocation-free form of disc_k_pass_a (the paper has no counterpart: this
 * exists for callers that cannot let a library allocate device memory, such
 * as applications that own all device memory through their own pool or run
 * under a fixed memory budget, and hosts that forbid plug-ins from calling
 * cudaMalloc or the stream-ordered allocator).  Same computation and outputs
 * as disc_k_pass_a, except that m_out is required (it receives m and is the
 * working buffer the moment pass reads), and that it always runs the 32 x 16
 * tiling (on volumes large enough for disc_k_pass_a's wide-tile pass, m, d and
 * u are the same bits but the norms may differ in their last bits: their float
 * partial sums are grouped by other CTAs).  The only scratch, the per-CTA norm
 * partial sums, lives in a fixed 64 KiB __device__ array inside the library,
 * present on every device that loads it until the process exits; launches
 * that would need more than 8192 CTAs (roughly, planes larger than about
 * 2048 x 2048 voxels) are rejected with DISC_ERR_SHAPE before any work is
 * queued.  The first call on each device looks up the array's device address
 * and caches it for the life of the process (call it once before any stream
 * capture).  The cached address does not survive cudaDeviceReset: a process
 * that resets a device must not call this entry point on it again.  All calls
 * share the array: calls whose work overlaps on the GPU race on it. */
disc_status disc_k_pass_a_static(const float* Im, const float* zs, const float* r,
                                 float* u, float* m_out, float* d_out,
                                 double* norms_out, int32_t nx, int32_t ny, int32_t nz,
                                 const int32_t patch[3], float qscale, float var_floor,
                                 int32_t force_mode, void* stream);

/* Gaussian regularisation (Algorithm A1 step 6, Sec. 2.3 kernel 2): each
 * component of u [3][nz][ny][nx] smoothed separably with taps
 * exp(-i^2 / 2 sigma^2), |i| <= radius (0 = ceil(3 sigma)), weights
 * renormalised over in-volume taps per axis; result in r.  r must not
 * alias u. */
disc_status disc_k_gauss(const float* u, float* r, int32_t nx, int32_t ny, int32_t nz,
                         float sigma, int32_t radius, void* stream);

/* The CBCT normalisation of disc_k_static_norm, and sd = STD(S) per voxel
 * (0 where Var(S) <= var_floor): the static patch statistics the mask of
 * Eq. 7 needs.  sd may be NULL. */
disc_status disc_k_static_stats(const float* Is, float* zs, float* sd, int32_t nx, int32_t ny,
                                int32_t nz, const int32_t patch[3], float qscale, float var_floor,
                                void* stream);

/* a_m of Sec. 2.3: the median of a = STD(M)/STD(S) (Eq. 5) over the voxels
 * with STD(S) > 0, for the image m (m = I_m for r = 0), with zs and sd from
 * disc_k_static_stats.  a_work (N floats, caller-owned) receives a, -1 where
 * STD(S) = 0.  *median_out (device double) receives the mean of the lower and
 * upper medians, -1 if no voxel qualifies. */
disc_status disc_k_ratio_median(const float* m, const float* zs, const float* sd, float* a_work,
                                double* median_out, int32_t nx, int32_t ny, int32_t nz,
                                const int32_t patch[3], float qscale, float var_floor, void* stream);

/* Algorithm A1 steps 1-3 with the mask: for the warped image m, a and b of
 * Eqs. 5-6, the mask xi of Eq. 7 (thresholds hu0, a_min, a_max) and the fill
 * of Eqs. 8-10 (box fill_t, weight scale fill_h, at most fill_passes Jacobi
 * passes).  Outputs (N each, caller-owned): a, b; d = I'_s - m with
 * I'_s = a I_s + b; stamp = 0 where xi = 0, the pass that filled the voxel, or
 * -1.  *remaining_out (device int32, may be NULL): voxels left unfilled. */
disc_status disc_k_correct_masked(const float* m, const float* Is, const float* zs, const float* sd,
                                  float* a, float* b, float* d, int32_t* stamp, int32_t* remaining_out,
                                  int32_t nx, int32_t ny, int32_t nz, const int32_t patch[3],
                                  float qscale, float var_floor, float hu0, float a_min, float a_max,
                                  float fill_h, const int32_t fill_t[3], int32_t fill_passes,
                                  void* stream);

/* Demons force (Eq. 1, Algorithm A1 steps 4-5) from d = I'_s - m and m:
 * grad I'_s = grad d + grad m by the path's differences, u = r + dr;
 * norms_out (device double[2], may be NULL): sum |dr|, sum |r|. */
disc_status disc_k_force(const float* m, const float* d, const float* r, float* u, double* norms_out,
                         int32_t nx, int32_t ny, int32_t nz, int32_t force_mode, void* stream);

/* ---------------------------------------------------------------------
 * Evaluation metrics (Sec. 2.4.3), between two images; not part of the
 * iteration.
 * ------------------------------------------------------------------- */

/* Normalised mutual information 2 I(A;B) / (H(A) + H(B)) in [0, 1] from a
 * joint histogram of `bins` (2..128) bins per image over each image's
 * [min, max] (bin = floor((v - min) * bins / (max - min)), in float32);
 * 1 when both images are constant.  *nmi_out: device double. */
disc_status disc_k_nmi(const float* a, const float* b, int64_t n, int32_t bins, double* nmi_out,
                       void* stream);

/* Binary Canny edge image (edges: N bytes, 1 = edge), slice by slice in z:
 * Gaussian smoothing (sigma, taps |i| <= ceil(3 sigma) <= 16, renormalised at
 * the borders), central-difference gradient, non-maximum suppression along
 * the gradient direction quantised to 45 degrees (a pixel needs M above
 * 1e-5 max|slice|), strong pixels M >= t_high max_slice(M), weak ones
 * M >= t_low times that, hysteresis over 8-connected weak pixels.  Every
 * decision is taken in float32 with explicitly rounded operations.
 * Synchronises `stream`. */
disc_status disc_k_canny(const float* img, uint8_t* edges, int32_t nx, int32_t ny, int32_t nz,
                         float sigma, float t_low, float t_high, void* stream);

/* Eq. (11): sqrt(sum_i (E1(i) - E2(i))^2 / N) of two binary edge images
 * (bytes, non-zero = edge).  *out: device double. */
disc_status disc_k_edge_rmse(const uint8_t* e1, const uint8_t* e2, int64_t n, double* out, void* stream);

/* Error word of the kernel-level calls above.  Their moment passes read
 * the volume through bulk tensor copies completed on shared-memory
 * barriers; a wait for such a copy is bounded (about one second), and one
 * that gives up abandons its tile and sets a device-wide error word instead
 * of hanging.  This call synchronises `stream`, returns DISC_ERR_TIMEOUT if
 * the word is set (and clears it), else DISC_OK.  (Registration and batch
 * contexts keep their own word and report DISC_ERR_TIMEOUT themselves at
 * their next synchronising call.)  The paper has no counterpart: it is the
 * failure report of this implementation's bounded waits. */
disc_status disc_k_check_error(void* stream);

/* ---------------------------------------------------------------------
 * Test switches (the paper has no counterpart).  Process-wide bits that
 * select the alternative paths the test suite compares against the default
 * ones, and failure hooks that need no GPU fault:
 *   DISC_SW_NO_TMA          moment passes read through per-thread loads
 *                           instead of bulk tensor copies (same results);
 *   DISC_SW_TMA_STALL       the bulk-copy-fed iteration pass arms its first
 *                           copy group for 16 bytes no copy delivers, so its
 *                           bounded wait gives up (about 1 s) and the call
 *                           reports DISC_ERR_TIMEOUT;
 *   DISC_SW_NO_GRAPH        contexts created afterwards launch each kernel on
 *                           the stream instead of replaying CUDA graphs;
 *   DISC_SW_UNROLLED_GRAPH  contexts created afterwards use unrolled graphs
 *                           even with a stop rule;
 *   DISC_SW_FAULT_ALLOC     disc_set_images's first device allocation reports
 *                           out-of-memory (host-side fault injection);
 *   DISC_SW_SEPARATE_WARP   contexts created afterwards warp I_m for the next
 *                           iteration in a kernel of its own after the
 *                           Gaussian at every level (same results);
 *   DISC_SW_FUSED_WARP      ... inside the Gaussian's xy pass at every level
 *                           (the default; in a batch it also keeps the
 *                           tuner from choosing the separate kernel);
 *   DISC_SW_WIDE_ANY        iteration passes planned afterwards take the
 *                           wide-tile kernel wherever it applies, whatever the
 *                           volume's size (same results; the planner otherwise
 *                           keeps it for volumes large enough to fill the GPU).
 * The initial bits come from the environment (DISC_NO_TMA, DISC_TEST_TMA_STALL,
 * DISC_NO_GRAPH, DISC_UNROLLED_GRAPH, DISC_WIDE_ANY, DISC_SEPARATE_WARP,
 * DISC_FUSED_WARP set to a non-zero value;
 * DISC_FAULT=alloc),
 * read once when the library is loaded.  disc_set_test_switches replaces all
 * bits; *previous (may be NULL) receives the old ones.  DISC_ERR_ARG for an
 * unknown bit.  Not synchronised with work in flight: change the switches
 * between calls, not during one. */
enum {
  DISC_SW_NO_TMA = 1,
  DISC_SW_TMA_STALL = 2,
  DISC_SW_NO_GRAPH = 4,
  DISC_SW_UNROLLED_GRAPH = 8,
  DISC_SW_FAULT_ALLOC = 16,
  DISC_SW_WIDE_ANY = 32,
  DISC_SW_SEPARATE_WARP = 64,
  DISC_SW_FUSED_WARP = 128,
  DISC_SW_ALL = 255
};
disc_status disc_set_test_switches(uint32_t flags, uint32_t* previous);

/* Bounds-checked build (the paper has no counterpart; the memory-safety check
 * of the test suite): a library compiled with -DDISC_BOUNDS_CHECK tests every
 * global index of the per-iteration kernels (warp, moment/force passes,
 * Gaussian passes, pyramid up- and down-sampling) against its buffer's extent
 * before the access; an index out of range is not accessed (loads read 0,
 * stores are dropped) and is counted on the device, never trapped.  This call
 * synchronises `stream`, returns the count recorded since the last call in
 * *count and clears it; *checked_build (may be NULL) receives 1 for such a
 * build.  In the normal build *count and *checked_build are 0. */
disc_status disc_bounds_violations(void* stream, int64_t* count, int32_t* checked_build);

#ifdef __cplusplus
}
#endif
#endif /* DISC_H */
