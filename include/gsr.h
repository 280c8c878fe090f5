/*
 * gsr.h - C ABI of the GB300 differentiable tile-based Gaussian rasterizer.
 *
 * The library renders 3D Gaussians (Sec. 3.1, Eq. 1: mean mu, covariance R S S^T R^T from a
 * quaternion and a scale, colour from spherical harmonics, opacity) into one or several posed
 * pinhole cameras by front-to-back alpha blending (Sec. 3.1, Eq. 2), returns RGB, accumulated
 * depth and expected depth (the rendered depth of the depth regulariser, Sec. 3.5.3) and opacity,
 * differentiates the blend with respect to every Gaussian parameter and a per-image 3x4 colour
 * transform, and selects per-partition detail levels by camera distance (Sec. 3.4.2).
 *
 * Conventions (one reading each where the paper is silent):
 *   - cameras: world->camera [R|t] 3x4 row-major, OpenCV axes (+x right, +y down, +z forward);
 *     pixel (x, y) samples the image point (x + 0.5, y + 0.5); mean2d = (fx X/Z + cx, fy Y/Z + cy).
 *   - projection: Sigma2D = J W Sigma W^T J^T + eps2d I, the Jacobian evaluated at X/Z, Y/Z clamped
 *     to +-1.3 (W/2)/fx and +-1.3 (H/2)/fy; with antialiased = 1 the opacity is multiplied by
 *     sqrt(det(J W Sigma W^T J^T) / det(Sigma2D)) (Sec. 3.5.4, Mip-Splatting 2D filter).
 *   - extent: r = ceil(3 sqrt(lambda_max)), lambda_max = m + sqrt(max(0.1, m^2 - det)); a Gaussian
 *     covers the 16x16 tiles [floor((mx - r)/16), floor((mx + r + 15)/16)) (same in y), clamped
 *     to the image; it never contributes outside those tiles.
 *   - tile culling (tile_cull = 1, Sec. 3.4.2 StopThePop): a (tile, Gaussian) pair is dropped
 *     when o' exp(-d2/2) < 1/255, d2 the smallest Mahalanobis distance from the mean to the
 *     rectangle of the tile's in-image pixel centres. Images are unchanged by the flag.
 *   - blending: alpha = min(0.99, o' exp(-sigma)); a Gaussian is skipped where sigma < 0 or
 *     alpha < 1/255; a pixel stops before the Gaussian that would take T below 1e-4.
 *   - order: by view-space depth z of the mean (FP32), ties to the lower Gaussian index.
 *   - colour: rgb = max(0, sum_k sh_k Y_k(dir) + 0.5), dir = normalize(mu - camera centre),
 *     real SH of degree <= 3 with Condon-Shortley phase, index l*l + l + m.
 *   - outputs per pixel: rgb = A C + b (1 - T) + T bg, where C = sum c_i alpha_i T_i and [A|b] the
 *     camera's appearance transform (identity when NULL); depth_acc = sum z_i alpha_i T_i;
 *     depth_exp = depth_acc / max(1 - T, 1e-10); alpha = 1 - T.
 *
 * Memory: every array argument marked "device" is caller-owned device memory on the context's
 * device, read-only unless it is an output. Outputs are overwritten, never accumulated. All
 * calls are asynchronous on `stream` except where stated; gsr_render_forward synchronises the
 * stream once (to size its pair buffers). A context is not thread-safe; use one per stream.
 * No exception and no abort crosses this ABI: every failure is a gsr_status.
 */
#ifndef GSR_H_
#define GSR_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* cudaStream_t-compatible handle; NULL is the legacy default stream. */
typedef struct CUstream_st* gsr_stream;

typedef enum gsr_status {
  GSR_OK = 0,
  GSR_WARN_OVER_BUDGET = 1,     /* gsr_select_lod: still over budget with every level at 0 */
  GSR_ERR_INVALID_ARG = -1,     /* a null pointer, a negative size, a value out of range */
  GSR_ERR_OOM = -2,             /* device allocation failed (context stays usable) */
  GSR_ERR_CUDA = -3,            /* a CUDA runtime call failed; see gsr_last_error */
  GSR_ERR_DEVICE_TIMEOUT = -4,  /* a bounded device wait ran out; results are invalid */
  GSR_ERR_UNSUPPORTED = -5      /* a size beyond what this build handles */
} gsr_status;

typedef enum gsr_dtype { GSR_F32 = 0, GSR_F16 = 1, GSR_BF16 = 2 } gsr_dtype;

typedef struct gsr_segment {
  int64_t begin; /* first Gaussian of the segment in the arrays */
  int64_t count; /* number of Gaussians */
} gsr_segment;

/* Per-Gaussian appearance transform (Sec. 3.5.1): each Gaussian has an embedding l_G (16) and
 * each image an embedding l_I (32); one hidden layer of 32 with ReLU and an output layer of 4
 * with a sigmoid (the sizes the paper gives) map [l_G ; l_I] to out. The paper says only that
 * out adjusts the Gaussian's colour and opacity (and pulls the opacity part toward zero); read
 * here as rgb' = 2 out[0..2] * rgb (the SH colour after its clamp; identity at 1/2) and
 * opacity' = (1 - out[3]) * opacity (after the anti-aliasing compensation; identity at 0).
 * All device memory, FP32, read-only; evaluated in FP32 per visible (Gaussian, camera). */
typedef struct gsr_appearance_mlp {
  const float* gauss_embed;  /* [n,16], indexed like the Gaussian arrays */
  const float* image_embed;  /* [n_cams,32]: one per camera of the launch, in camera order */
  const float* params;       /* [1700]: w1 [32][48] | b1 [32] | w2 [4][32] | b2 [4], row-major;
                                hidden = ReLU(w1 [l_G ; l_I] + b1), out = sigmoid(w2 hidden + b2) */
  /* Or, for rendering only: the outputs [n,4] of every Gaussian for one image embedding, from
   * gsr_appearance_cache (16-byte aligned). When set, the three arrays above are not read, every
   * camera of the launch uses these outputs, and gsr_render_backward refuses the struct. */
  const float* cached;
} gsr_appearance_mlp;

/* Gaussians (Sec. 3.1, Eq. 1), structure of arrays, all device memory.
 * If segs != NULL only the listed segments are rendered, in list order (the order decides the
 * index used for depth ties); segs is HOST memory with nsegs entries.
 * seg_cams (HOST, nsegs entries, or NULL = every camera renders every segment): bit c set means
 * camera c of the launch renders segment k. A launch can so render several views whose detail
 * levels differ (Sec. 3.4.2: a level per partition and per view): the segments are the union
 * of the views' selections, each marked with the views that selected it. A camera's images are
 * then those of rendering its own segments alone, in the same relative order. */
typedef struct gsr_gaussians {
  int64_t n;              /* number of Gaussians in the arrays */
  const float* means;     /* [n,3] float32, world coordinates */
  const void* scales;     /* [n,3] attr_dtype, linear standard deviations (> 0) */
  const void* quats;      /* [n,4] attr_dtype, (w, x, y, z), need not be normalised */
  const void* opacities;  /* [n] attr_dtype, in [0, 1] */
  const void* sh;         /* [n, sh_coeffs, 3] sh_dtype, coefficient-major, RGB innermost */
  int32_t sh_coeffs;      /* coefficients stored per Gaussian, (sh_degree+1)^2 <= sh_coeffs <= 16 */
  int32_t sh_degree;      /* 0..3 */
  int32_t attr_dtype;     /* gsr_dtype of scales, quats, opacities */
  int32_t sh_dtype;       /* gsr_dtype of sh */
  const gsr_segment* segs;
  int32_t nsegs;
  const gsr_appearance_mlp* mlp;  /* appearance transform (HOST struct, device arrays), or NULL */
  const uint32_t* seg_cams;       /* [nsegs] camera masks of the segments (HOST), or NULL */
} gsr_gaussians;

/* One pinhole camera (host memory). */
typedef struct gsr_camera {
  float viewmat[12];       /* world->camera [R|t], row-major 3x4 */
  float fx, fy, cx, cy;    /* pixels; fx, fy > 0 */
  int32_t width, height;   /* 1..16384 */
  float near_plane;        /* > 0 (0.01 by convention) */
  float far_plane;         /* > near_plane (1e10 by convention) */
  const float* appearance; /* device [3,4] row-major [A|b] applied to each Gaussian colour, or NULL */
} gsr_camera;

typedef struct gsr_opts {
  float eps2d;          /* low-pass dilation in px^2 (0.3) */
  int32_t antialiased;  /* 1: opacity compensation of the 2D filter (Sec. 3.5.4) */
  int32_t tile_cull;    /* 1: StopThePop tile culling (Sec. 3.4.2) */
  float bg[3];          /* background colour blended with the final transmittance */
  int32_t save_state;   /* 1: keep sorted pairs for backward; 0: backward recomputes them */
  int32_t absgrad;      /* 1: backward also accumulates sum |dL/dmean2d| per axis (AbsGS) */
  int32_t global_sort;  /* how the (tile, Gaussian) pairs are put in (tile, depth, index) order:
                           0 (default): counted per tile, placed in each tile's range and sorted per
                           tile in shared memory; 1: the visible records sorted by depth and the
                           pairs sorted stably by tile with the onesweep radix sort. Same order,
                           same results; only the timing differs. */
} gsr_opts;

/* Forward outputs, device float32, cameras packed one after another (camera c starts at pixel
 * sum_{c'<c} W H), row-major within a camera. rgb is required; the others may be NULL. */
typedef struct gsr_outputs {
  float* rgb;        /* [P,3] */
  float* depth_acc;  /* [P] */
  float* depth_exp;  /* [P] */
  float* alpha;      /* [P] */
} gsr_outputs;

/* Upstream gradients dL/d(output), same layout as gsr_outputs; NULL means zero. */
typedef struct gsr_out_grads {
  const float* rgb;
  const float* depth_acc;
  const float* depth_exp;
  const float* alpha;
} gsr_out_grads;

/* Parameter gradients, device float32, overwritten. Rows not rendered (outside the segments,
 * culled in every camera) are set to zero. appearance and absgrad may be NULL. */
typedef struct gsr_param_grads {
  float* means;       /* [n,3] */
  float* scales;      /* [n,3] */
  float* quats;       /* [n,4] */
  float* opacities;   /* [n] */
  float* sh;          /* [n, sh_coeffs, 3] */
  float* appearance;  /* [C,3,4] (cameras without appearance get the gradient of the identity) */
  float* absgrad;     /* [n,2] sum over pixels and cameras of |dL/dmean2d_x|, |dL/dmean2d_y| */
  /* appearance transform (required when g->mlp != NULL, ignored otherwise): */
  float* gauss_embed; /* [n,16] */
  float* image_embed; /* [C,32] */
  float* mlp_params;  /* [1700], laid out like gsr_appearance_mlp.params */
} gsr_param_grads;

/* Optional device allocator (e.g. a framework's caching allocator). NULL: cudaMalloc/cudaFree. */
typedef struct gsr_allocator {
  void* (*alloc)(size_t bytes, gsr_stream stream, void* user);
  void (*free)(void* ptr, size_t bytes, gsr_stream stream, void* user);
  void* user;
} gsr_allocator;

typedef struct gsr_ctx gsr_ctx;
typedef struct gsr_fwd_state gsr_fwd_state;

/* Sizes recorded by a forward pass. */
typedef struct gsr_state_info {
  int64_t n_render;   /* Gaussians rendered (sum of segment counts, or n) */
  int32_t n_cams;
  int64_t n_visible;  /* V: visible (camera, Gaussian) pairs */
  int64_t n_pairs;    /* P: (tile, Gaussian) pairs after culling */
  int64_t n_tiles;    /* sum over cameras of tiles_x * tiles_y */
  int64_t n_pixels;   /* sum over cameras of W * H */
  int64_t max_tile_pairs;  /* pairs of the fullest tile */
} gsr_state_info;

/* Buffers of a forward state that gsr_state_copy can export (for tests and tools). */
typedef enum gsr_state_buffer {
  GSR_BUF_RECORDS = 0,    /* [V] 64-byte splat records (float4 x4: mean2d, opacity', z | conic, red |
                             green, blue, packed tile rectangle and camera | alpha >= 1/255 box) */
  GSR_BUF_OWNER = 1,      /* [V] uint32: rendered index of each record's Gaussian; a Gaussian's
                             records are consecutive, in camera order */
  GSR_BUF_PAIR_VALS = 2,  /* [P] uint32 record index, sorted by (tile, depth, index) */
  GSR_BUF_RANGES = 3,     /* [n_tiles] uint32 x2: [start, end) into the pair list */
  GSR_BUF_T_FINAL = 4,    /* [n_pixels] float32 final transmittance */
  GSR_BUF_N_CONTRIB = 5,  /* [n_pixels] uint32 list positions walked up to the last contributor */
  GSR_BUF_DEPTH_STATE = 6 /* [n_pixels] float32 x2: depth of the pixel's first contributor z_f, and
                             sum over contributors of (z - z_f) alpha T (depth_acc = z_f (1 - T) + it) */
} gsr_state_buffer;

/* ---- context --------------------------------------------------------------------------- */

/* Creates a context on `device` (cudaSetDevice is called). alloc may be NULL. */
gsr_status gsr_create(gsr_ctx** out, int device, const gsr_allocator* alloc);
/* Frees the context's workspace; states created from it must be released first. */
void gsr_destroy(gsr_ctx* ctx);
const char* gsr_status_string(gsr_status s);
/* Text of the last error on this context ("" if none). */
const char* gsr_last_error(const gsr_ctx* ctx);
/* Bytes of workspace the last forward of this size would hold (for admission by memory). */
gsr_status gsr_workspace_query(gsr_ctx* ctx, int64_t n_render, const gsr_camera* cams, int32_t n_cams,
                               int64_t expected_pairs, size_t* bytes_out);
/* Bytes currently held by the context (workspace only, not states). */
size_t gsr_workspace_bytes(const gsr_ctx* ctx);

/* ---- rendering ------------------------------------------------------------------------- */

/* Forward pass (Sec. 3.1, Eq. 2) of n_cams cameras (1..32) in one launch sequence.
 * state_out: if non-NULL, receives a state (owned by ctx, released with gsr_state_release)
 * that gsr_render_backward needs. Synchronises `stream` once, after binning. */
gsr_status gsr_render_forward(gsr_ctx* ctx, const gsr_gaussians* g, const gsr_camera* cams, int32_t n_cams,
                              const gsr_opts* opts, const gsr_outputs* out, gsr_fwd_state** state_out,
                              gsr_stream stream);

/* Backward pass: gradients of L given dL/d(outputs). g, cams, n_cams and opts must be those of
 * the forward that produced `state`, with the same array contents. Every gradient array of
 * `grads` is overwritten (not accumulated into); rows of Gaussians without a record are zero.
 * With g->mlp set, grads->gauss_embed, image_embed and mlp_params are required and receive the
 * appearance transform's gradients (Sec. 3.5.1); the records' opacity and colour gradients are
 * carried through the transform before the projection backward. Asynchronous. Errors:
 * GSR_ERR_INVALID_ARG (null or mismatched inputs, a null gradient array), GSR_ERR_OOM,
 * GSR_ERR_CUDA, GSR_ERR_DEVICE_TIMEOUT (recompute mode: a bounded wait of the re-run binning). */
gsr_status gsr_render_backward(gsr_ctx* ctx, const gsr_gaussians* g, const gsr_camera* cams, int32_t n_cams,
                               const gsr_opts* opts, const gsr_fwd_state* state, const gsr_out_grads* dout,
                               const gsr_param_grads* grads, gsr_stream stream);

/* Zeroes the parameter-gradient arrays of `grads` (means, scales, quats, opacities, sh and, when
 * not NULL, absgrad and, with g->mlp set, gauss_embed; sized for g->n Gaussians and g->sh_coeffs
 * as in gsr_render_backward; the backward zeroes the small image_embed and mlp_params itself) ahead
 * of the backward pass. No counterpart in the paper. The call records the request (a fill still
 * queued for an earlier request is ordered before later work on `stream`; nothing else is
 * queued): the next gsr_render_backward on this context that is given exactly these arrays
 * queues this memory-bound fill (236 bytes per Gaussian in FP32) on the context's internal
 * stream right before its blend, which it runs beside, and waits for it before writing the
 * rows; that is also what a backward does without a request, so the request only fixes the
 * arrays ahead of time. (Queuing the fill earlier, at the end of the forward, was measured
 * slower: started alone it then shared the GPU badly with the blend backward.) A backward given
 * other arrays zeroes the requested ones too, ordered before everything it queues after, and
 * fills its own. The caller must not use the arrays between
 * this call and that backward. Errors: GSR_ERR_INVALID_ARG (null struct or gradient array). */
gsr_status gsr_param_grads_zero(gsr_ctx* ctx, const gsr_gaussians* g, const gsr_param_grads* grads,
                                gsr_stream stream);

void gsr_state_release(gsr_ctx* ctx, gsr_fwd_state* state);
gsr_status gsr_state_get_info(const gsr_fwd_state* state, gsr_state_info* info);
/* Copies `bytes` of a state buffer into device memory `dst` (stream-ordered). */
gsr_status gsr_state_copy(const gsr_fwd_state* state, int32_t which, void* dst, size_t bytes,
                          gsr_stream stream);

/* Waits for `stream` and reports any error recorded by a bounded device wait since the last
 * forward began (GSR_ERR_DEVICE_TIMEOUT), then clears it. */
gsr_status gsr_sync_check(gsr_ctx* ctx, gsr_stream stream);

/* Pace of the gradient zero fill (no counterpart in the paper). The fill of the parameter-gradient
 * arrays (gsr_param_grads_zero, or the backward's own) runs on the context's side stream beside the
 * backward's blend; at full speed it takes most of the memory bandwidth from the stages it
 * overlaps. gb_per_s > 0 spreads it out at about that rate (each fill block starts a 16 KB chunk
 * only when it is due on the GPU's nanosecond timer); 0 writes as fast as possible. The default,
 * 5600 GB/s, is just under what the fill reaches alone on a GB300; so paced, it leaves the blend
 * backward beside it its memory latency (measured on a 6M-Gaussian 1080p step: 730 us against
 * 776 unpaced). blocks > 0 sets how many blocks fill (0 keeps the current number; the default is
 * one per SM).
 * Results are the same either way; only the timing changes. Errors: GSR_ERR_INVALID_ARG. */
gsr_status gsr_set_fill_rate(gsr_ctx* ctx, float gb_per_s, int32_t blocks);

/* Where a requested gradient fill (gsr_param_grads_zero) runs (no counterpart in the paper).
 * The parameter-gradient rows of every Gaussian are zeroed each backward (236 bytes per Gaussian
 * in FP32, memory-bound) by a small kernel on the context's side stream. The first early_share
 * of a requested fill's bytes (in the arrays' order: means, scales, quats, opacities, sh,
 * absgrad, gauss_embed) is queued by the next forward right after its preprocess, beside the
 * binning and the forward blend; the rest by the backward right before its blend, beside it.
 * 0 (the default, measured fastest on a 6M-Gaussian 1080p scene) queues all of it with the
 * backward. Results are the same either way; only the timing changes. Errors:
 * GSR_ERR_INVALID_ARG (outside [0, 1]). */
gsr_status gsr_set_fill_split(gsr_ctx* ctx, float early_share);

/* Failure detection (no counterpart in the paper). Every device wait of this context's kernels
 * (the decoupled look-backs of the chained scans and of the sort) gives up after `polls` polls
 * (0: the default, 2^20, well under a second), sets the context's error word and lets the kernel
 * finish; the call that checks the word (gsr_render_forward, a recompute-mode
 * gsr_render_backward, gsr_sync_check) returns GSR_ERR_DEVICE_TIMEOUT and the results of that
 * call are invalid, while every write stays inside its buffers. never_ready = 1 is a test switch:
 * every look-back then treats its predecessors' status words as unpublished, so each wait runs to
 * its limit (a wait on a flag nothing sets). The context stays usable: setting (0, 0) restores
 * normal operation. Host-side only; takes effect from the next call. */
gsr_status gsr_set_wait_limit(gsr_ctx* ctx, uint32_t polls, int32_t never_ready);

/* Evaluates the appearance transform (Sec. 3.5.1) of every Gaussian of g (array order, segments
 * ignored) for the image embedding in row `image` of g->mlp->image_embed, into out [g->n,4]
 * (device memory, 16-byte aligned). The paper notes that these offsets can be kept while the
 * image embedding is unchanged; passing them as g->mlp->cached renders without evaluating the
 * transform, with the same bits as evaluating it for a camera with that embedding. Needs
 * g->mlp's gauss_embed, image_embed and params; `image` must be a row of image_embed.
 * Asynchronous. Errors: GSR_ERR_INVALID_ARG (null or misaligned arrays, image < 0). */
gsr_status gsr_appearance_cache(gsr_ctx* ctx, const gsr_gaussians* g, int32_t image, float* out, gsr_stream stream);

/* ---- profiling ------------------------------------------------------------------------- */

/* Stages timed with CUDA events on the call's stream while profiling is on. */
typedef enum gsr_stage {
  GSR_STAGE_PREPROCESS = 0,     /* projection, colour, cull, compaction */
  GSR_STAGE_TILE_COUNT = 1,     /* (tile, record) pairs counted per tile (global_sort: per record,
                                   with tile culling only) */
  GSR_STAGE_TILE_SCAN = 2,      /* scan of the tile counts: each tile's range of pairs, P (global_sort:
                                   of the records' counts in depth order: their pair offsets, P) */
  GSR_STAGE_READBACK = 3,       /* the forward's one device-to-host read of V and P */
  GSR_STAGE_PLACE = 4,          /* pairs written into their tiles' ranges (global_sort: at their
                                   records' offsets, keyed by tile) */
  GSR_STAGE_TILE_SORT = 5,      /* every tile's pairs sorted by (depth, index) (global_sort: the
                                   pairs sorted stably by tile) */
  GSR_STAGE_BLEND_FWD = 6,      /* forward compositing */
  GSR_STAGE_BLEND_BWD = 7,      /* backward compositing */
  GSR_STAGE_PREPROCESS_BWD = 8, /* projection and colour backward */
  GSR_STAGE_BETWEEN = 9,        /* idle time between consecutive stages of one call (memsets,
                                   waits on the host or the side stream, launch latency) */
  GSR_STAGE_APPEARANCE_BWD = 10,/* appearance-transform backward (only with gsr_gaussians.mlp) */
  GSR_STAGE_DEPTH_SORT = 11,    /* global_sort: radix sort of the visible records by depth */
  GSR_STAGE_RANGES = 12,        /* global_sort: each tile's range in the sorted pairs */
  GSR_NUM_STAGES = 13
} gsr_stage;

/* Counters gathered while profiling with count_evals = 1. */
typedef enum gsr_counter {
  GSR_CNT_FWD_EVALS = 0,     /* (pixel, Gaussian) evaluations in the forward blend */
  GSR_CNT_FWD_CONTRIBS = 1,  /* of which blended (alpha >= 1/255, before termination) */
  GSR_CNT_BWD_EVALS = 2,     /* (pixel, Gaussian) positions visited by the backward blend */
  GSR_CNT_BWD_CONTRIBS = 3,  /* of which contributors */
  GSR_CNT_BWD_WARP_ITERS = 4,          /* (warp, Gaussian) iterations the backward blend evaluates */
  GSR_CNT_BWD_WARP_ITERS_CONTRIB = 5,  /* of which at least one pixel of the warp takes the Gaussian */
  GSR_NUM_COUNTERS = 6
} gsr_counter;

/* on = 1 records CUDA events around every stage of later calls; count_evals = 1 also counts
 * blend evaluations (slightly slower kernels). */
gsr_status gsr_profile_enable(gsr_ctx* ctx, int32_t on, int32_t count_evals);
/* Restricts the recorded events to the stages whose bit is set in stage_mask (bit k = stage k;
 * all stages by default). Timing one kernel inside a longer loop this way adds two events per
 * launch instead of two per stage. GSR_STAGE_BETWEEN is only meaningful with all stages on. */
gsr_status gsr_profile_select(gsr_ctx* ctx, uint32_t stage_mask);
/* Waits for every recorded event, adds the elapsed milliseconds and launch counts of each stage
 * since the last collect into ms[GSR_NUM_STAGES] and launches[GSR_NUM_STAGES] (either may be
 * NULL), the counters into counters[GSR_NUM_COUNTERS] (may be NULL), then clears them. */
gsr_status gsr_profile_collect(gsr_ctx* ctx, double* ms, int64_t* launches, int64_t* counters);

/* ---- building blocks ------------------------------------------------------------------- */

/* Stable LSD radix sort of n (key, value) pairs of uint32 by key bits [begin_bit, end_bit),
 * 8 bits per pass, one chained-scan (onesweep) kernel per pass. keys_in/vals_in are not
 * modified; the result goes to keys_out/vals_out (device, must not alias the inputs).
 * n < 2^30. Uses the context's workspace. */
gsr_status gsr_sort_pairs_u32(gsr_ctx* ctx, const uint32_t* keys_in, const uint32_t* vals_in,
                              uint32_t* keys_out, uint32_t* vals_out, int64_t n, int32_t begin_bit,
                              int32_t end_bit, gsr_stream stream);

/* The sort of gsr_sort_pairs_u32 for callers that cannot allocate device memory: code being
 * recorded into a CUDA graph (an allocation cannot be captured, and cudaMalloc may
 * synchronise the device), a loop that must keep a fixed memory footprint, or a callback that
 * runs inside another framework's allocator. It calls no cudaMalloc, cudaFree or allocating
 * library routine. The paper has no counterpart: this is a deployment variant of the sort.
 *   Limit: n <= 262144 (2^18); a larger n returns GSR_ERR_UNSUPPORTED without doing anything.
 *   Scratch: one static device array of about 2.6 MB inside libgsr, reserved on every GPU that
 *     loads the library until the process exits and shared by every call. Calls that overlap
 *     on the GPU (two streams, or two host threads) race on it and give wrong results:
 *     serialise them on one stream. Each call clears what must start at zero (the look-back
 *     status words, the digit counts and the block counters) with stream-ordered memsets.
 *   The first call on a device looks up the array's device address with that device current
 *     and keeps it for the life of the process; make that first call before any stream
 *     capture. A process that calls cudaDeviceReset must not call this entry point again on
 *     that device (the kept address would be stale).
 *   device_err: required, device int32; a bounded wait that runs out ORs 1 into it (the output
 *     is then invalid); the call never clears it. NULL returns GSR_ERR_INVALID_ARG: a timeout
 *     must have somewhere to be reported.
 *   begin_bit == end_bit copies the inputs to the outputs.
 * Asynchronous on `stream`; inputs are not modified; outputs must not alias the inputs. */
gsr_status gsr_sort_pairs_u32_noalloc(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                                      uint32_t* vals_out, int64_t n, int32_t begin_bit, int32_t end_bit,
                                      int32_t* device_err, gsr_stream stream);

/* ---- detail levels (Sec. 3.4.2) -------------------------------------------------------- */

/* Partition-level detail-level selection for one camera, host memory throughout.
 *   aabb[P][6]: xmin, ymin, zmin, xmax, ymax, zmax of each partition (world).
 *   level_offsets[L][P+1]: Gaussians of partition p at level l occupy
 *     [level_offsets[l][p], level_offsets[l][p+1]) of the concatenated resident arrays;
 *     level 0 is the coarsest, L-1 the finest.
 *   thresholds[L-1], ascending: camera distance (to the closest point of the box) below
 *     thresholds[k] selects level L-1-k; at or above the last one, level 0.
 *   A partition is culled (level -1) when all 8 corners of its box are strictly outside one
 *     of the frustum's six half-spaces (near, far, the four image borders).
 *   budget > 0: while the selected total exceeds it, lower the farthest partition above level 0
 *     (ties: larger index) by one level; GSR_WARN_OVER_BUDGET if it cannot get under.
 * Outputs: levels[P]; segs[<= P] in partition order (empty ones skipped); *nsegs; *n_selected. */
gsr_status gsr_select_lod(int32_t P, const double* aabb, int32_t L, const int64_t* level_offsets,
                          const gsr_camera* cam, const double* thresholds, int64_t budget, int32_t* levels,
                          gsr_segment* segs, int32_t* nsegs, int64_t* n_selected);

#ifdef __cplusplus
}
#endif

#endif /* GSR_H_ */
