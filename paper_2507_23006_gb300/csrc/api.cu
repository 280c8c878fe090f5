// C ABI of libgsr: context, workspace, forward / backward orchestration, detail-level selection.
//
// Forward launch sequence on the caller's stream (Sec. 3.1, Eq. 2 and the tile-based binning):
//   preprocess (projection + colour + cull, compacted by a chained scan)
//   -> pair counts per tile -> chained scan over the tiles (each tile's range, P)
//   -> one stream synchronisation to read V and P and size the pair buffers
//   -> pairs placed in their tiles' ranges -> each tile's list sorted by (depth, index)
//   -> blend.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/gsr.h"
#include "gsr_internal.cuh"

using namespace gsr;

namespace {

struct Buf {
  void* p = nullptr;
  size_t cap = 0;
};

}  // namespace

struct gsr_ctx {
  int device = 0;
  gsr_allocator alloc{};
  bool has_alloc = false;
  std::string last_error;
  size_t held = 0;
  // scratch
  Buf seg_begin, seg_start, seg_cams;
  Buf rec, owner;                              // records (recompute / no-state mode)
  Buf rcam;                                    // camera of each record (preprocess passes)
  Buf sort_ktmp, sort_vtmp, sort_hist, sort_status;  // gsr_sort_pairs_u32
  Buf pre_vis, pre_counts, scan_status, misc, tile_ctr, big_tiles;
  Buf pair_keys, key_scratch, pvals_s, ranges;  // pairs (pvals_s, ranges: no-state mode)
  Buf dkeys, dvals, touched, dkeys_s, dvals_s, offsets, cnt_sorted, pkeys, pvals, pkeys_s;  // global sort
  Buf pix_T, pix_n, pix_D;                     // per-pixel state (no-state mode)
  Buf g2d, gaff;
  // host pinned staging of the binning counters (misc, 32 bytes) and the error word
  void* pinned = nullptr;
  int* d_err = nullptr;  // 64 bytes: error word at 0, blend counters (GSR_NUM_COUNTERS x u64) at byte 8
  // profiling
  bool prof = false;
  bool count_evals = false;
  struct Rec3 {
    int stage;
    cudaEvent_t a, b;
    uint64_t call;  // the API call that recorded it
  };
  uint64_t call_seq = 0;
  std::vector<Rec3> prof_recs;
  uint32_t prof_mask = 0xffffffffu;  // stages whose events are recorded (bit k = stage k)
  std::vector<cudaEvent_t> ev_pool;
  // released forward states kept with their buffers for reuse (stream-ordered, no sync)
  std::vector<gsr_fwd_state*> state_pool;
  uint32_t epoch = 0;  // tag of the chained-scan status words of the latest launch
  // a second stream for work that overlaps the caller's (joined back before returning)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_prezero = nullptr, ev_prezero_early = nullptr;
  FillSpans prezero{};           // gradient arrays to zero ahead (gsr_param_grads_zero)
  bool prezero_requested = false;  // recorded, the rest of the fill not queued yet
  bool prezero_pending = false;    // the rest queued (ev_prezero marks its end), not used yet
  bool prezero_early = false;      // the first part queued by a forward (ev_prezero_early marks its end)
  size_t prezero_queued = 0;       // floats of the requested fill queued so far
  int grid_cap = 304;  // resident blocks of the looping scan / sort kernels (2 per SM)
  int fill_blocks = 152;  // blocks of the gradient zero fill (one per SM)
  // pace of the gradient zero fill in GB/s (0: unpaced); gsr_set_fill_rate. Paced just under the
  // rate it reaches alone, the fill leaves the blend backward it runs beside its memory latency:
  // 730 us per step on the 6M city at 1080p against 776 unpaced (5000-6000 GB/s measured alike)
  float fill_gbs = 5600.f;
  float fill_early = 0.f;  // share of a requested fill queued after the forward's preprocess
  WaitCfg wait;  // how the look-backs of this context's kernels wait (gsr_set_wait_limit)
  // default allocator: a context-owned stream-ordered pool (growth and release never
  // synchronise the device, which matters when several contexts serve concurrently)
  cudaMemPool_t pool = nullptr;
  cudaStream_t last_stream = nullptr;
};

struct gsr_fwd_state {
  gsr_ctx* ctx = nullptr;
  gsr_state_info info{};
  bool has_bins = false;
  Buf rec, owner, pvals_s, ranges;
  Buf T_final, n_contrib, D;
};

namespace {

gsr_status set_err(gsr_ctx* ctx, gsr_status st, const char* msg) {
  if (ctx) ctx->last_error = msg ? msg : "";
  return st;
}

gsr_status cuda_err(gsr_ctx* ctx, cudaError_t e, const char* where) {
  if (e == cudaSuccess) return GSR_OK;
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  if (ctx) ctx->last_error = m;
  return e == cudaErrorMemoryAllocation ? GSR_ERR_OOM : GSR_ERR_CUDA;
}

void* raw_alloc(gsr_ctx* ctx, size_t bytes, cudaStream_t s) {
  if (bytes == 0) bytes = 16;
  if (ctx->has_alloc) return ctx->alloc.alloc(bytes, reinterpret_cast<gsr_stream>(s), ctx->alloc.user);
  void* p = nullptr;
  const cudaError_t e = ctx->pool ? cudaMallocFromPoolAsync(&p, bytes, ctx->pool, s) : cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void raw_free(gsr_ctx* ctx, void* p, size_t bytes, cudaStream_t s) {
  if (!p) return;
  if (ctx->has_alloc) ctx->alloc.free(p, bytes, reinterpret_cast<gsr_stream>(s), ctx->alloc.user);
  else if (ctx->pool) cudaFreeAsync(p, s);
  else cudaFree(p);
}

// Grows `b` to hold at least `bytes` (contents are not preserved).
bool ensure(gsr_ctx* ctx, Buf& b, size_t bytes, cudaStream_t s) {
  if (b.cap >= bytes && b.p) return true;
  if (b.p) {
    raw_free(ctx, b.p, b.cap, s);
    ctx->held -= b.cap;
    b.p = nullptr;
    b.cap = 0;
  }
  size_t want = std::max<size_t>(bytes + bytes / 2, 256);
  want = (want + 255) & ~static_cast<size_t>(255);
  b.p = raw_alloc(ctx, want, s);
  if (!b.p) return false;
  b.cap = want;
  ctx->held += want;
  return true;
}

void release(gsr_ctx* ctx, Buf& b, cudaStream_t s) {
  if (b.p) {
    raw_free(ctx, b.p, b.cap, s);
    ctx->held -= b.cap;
  }
  b.p = nullptr;
  b.cap = 0;
}

template <typename T>
T* as(Buf& b) {
  return static_cast<T*>(b.p);
}

// Like ensure(), but a new allocation is zeroed: status words of epoch 0 are never "ready".
bool ensure_zeroed(gsr_ctx* ctx, Buf& b, size_t bytes, cudaStream_t s) {
  const void* before = b.p;
  if (!ensure(ctx, b, bytes, s)) return false;
  if (b.p != before) cudaMemsetAsync(b.p, 0, b.cap, s);
  return true;
}

// A fresh tag for the status words of one chained-scan launch. After 2^30 - 1 tags the status
// arrays are cleared and the count restarts.
uint32_t next_epoch(gsr_ctx* ctx, cudaStream_t s) {
  if (++ctx->epoch >= (1u << 30)) {
    Buf* st[] = {&ctx->scan_status, &ctx->sort_status};  // every chained scan's words
    for (Buf* b : st)
      if (b->p) cudaMemsetAsync(b->p, 0, b->cap, s);
    ctx->epoch = 1;
  }
  return ctx->epoch;
}

SortScratch sort_scratch(gsr_ctx* ctx) {
  SortScratch sc;
  sc.keys_tmp = as<uint32_t>(ctx->sort_ktmp);
  sc.vals_tmp = as<uint32_t>(ctx->sort_vtmp);
  sc.hist = as<uint32_t>(ctx->sort_hist);
  sc.status = as<unsigned long long>(ctx->sort_status);
  sc.grid_cap = ctx->grid_cap;
  sc.wait = ctx->wait;
  return sc;
}

bool ensure_sort(gsr_ctx* ctx, long long n, cudaStream_t s) {
  const size_t words = sort_status_words(n) * 4;  // four passes at most
  return ensure(ctx, ctx->sort_ktmp, sizeof(uint32_t) * n, s) && ensure(ctx, ctx->sort_vtmp, sizeof(uint32_t) * n, s) &&
         ensure(ctx, ctx->sort_hist, sizeof(uint32_t) * kSortCountWords, s) &&
         ensure_zeroed(ctx, ctx->sort_status, sizeof(unsigned long long) * words, s);
}

unsigned long long* counters_of(gsr_ctx* ctx) {
  return ctx->count_evals ? reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(ctx->d_err) + 8) : nullptr;
}

cudaEvent_t take_event(gsr_ctx* ctx) {
  if (!ctx->ev_pool.empty()) {
    cudaEvent_t e = ctx->ev_pool.back();
    ctx->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Records CUDA events around one stage while profiling is on.
struct StageTimer {
  gsr_ctx* ctx;
  int stage;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  StageTimer(gsr_ctx* c, int st, cudaStream_t str) : ctx(c), stage(st), s(str) {
    if (ctx->prof && ((ctx->prof_mask >> st) & 1u) && (a = take_event(ctx))) cudaEventRecord(a, s);
  }
  ~StageTimer() {
    if (!a) return;
    cudaEvent_t b = take_event(ctx);
    if (!b) {
      ctx->ev_pool.push_back(a);
      return;
    }
    cudaEventRecord(b, s);
    ctx->prof_recs.push_back({stage, a, b, ctx->call_seq});
  }
};

bool finite3x4(const float* v) {
  for (int i = 0; i < 12; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

gsr_status validate(gsr_ctx* ctx, const gsr_gaussians* g, const gsr_camera* cams, int32_t C, const gsr_opts* o) {
  if (!ctx) return GSR_ERR_INVALID_ARG;
  if (!g || !cams || !o) return set_err(ctx, GSR_ERR_INVALID_ARG, "null gaussians, cameras or opts");
  if (C < 1 || C > kMaxCams) return set_err(ctx, GSR_ERR_INVALID_ARG, "n_cams must be in 1..32");
  if (g->n < 0) return set_err(ctx, GSR_ERR_INVALID_ARG, "negative n");
  if (g->n > 0 && (!g->means || !g->scales || !g->quats || !g->opacities || !g->sh))
    return set_err(ctx, GSR_ERR_INVALID_ARG, "null Gaussian array with n > 0");
  if (g->sh_degree < 0 || g->sh_degree > 3) return set_err(ctx, GSR_ERR_INVALID_ARG, "sh_degree must be 0..3");
  if (g->sh_coeffs < (g->sh_degree + 1) * (g->sh_degree + 1) || g->sh_coeffs > 16)
    return set_err(ctx, GSR_ERR_INVALID_ARG, "sh_coeffs must be in (deg+1)^2..16");
  if (g->attr_dtype < 0 || g->attr_dtype > 2 || g->sh_dtype < 0 || g->sh_dtype > 2)
    return set_err(ctx, GSR_ERR_INVALID_ARG, "unknown dtype");
  if (g->nsegs < 0 || (g->nsegs > 0 && !g->segs)) return set_err(ctx, GSR_ERR_INVALID_ARG, "bad segment list");
  if (g->seg_cams && !g->segs) return set_err(ctx, GSR_ERR_INVALID_ARG, "segment camera masks without segments");
  if (g->mlp && !g->mlp->cached && (!g->mlp->image_embed || !g->mlp->params || (g->n > 0 && !g->mlp->gauss_embed)))
    return set_err(ctx, GSR_ERR_INVALID_ARG, "null appearance-transform array");
  if (g->mlp && g->mlp->cached && reinterpret_cast<uintptr_t>(g->mlp->cached) % 16 != 0)
    return set_err(ctx, GSR_ERR_INVALID_ARG, "cached appearance outputs must be 16-byte aligned");
  for (int s = 0; s < g->nsegs; ++s) {
    const gsr_segment& sg = g->segs[s];
    if (sg.begin < 0 || sg.count < 0 || sg.begin + sg.count > g->n)
      return set_err(ctx, GSR_ERR_INVALID_ARG, "segment outside the arrays");
  }
  for (int c = 0; c < C; ++c) {
    const gsr_camera& k = cams[c];
    if (!(k.fx > 0.f) || !(k.fy > 0.f) || !std::isfinite(k.fx) || !std::isfinite(k.fy))
      return set_err(ctx, GSR_ERR_INVALID_ARG, "fx, fy must be positive");
    if (k.width < 1 || k.height < 1 || k.width > 16384 || k.height > 16384)
      return set_err(ctx, GSR_ERR_INVALID_ARG, "width and height must be in 1..16384");
    if (!(k.near_plane > 0.f) || !(k.far_plane > k.near_plane))
      return set_err(ctx, GSR_ERR_INVALID_ARG, "need 0 < near < far");
    if (!finite3x4(k.viewmat) || !std::isfinite(k.cx) || !std::isfinite(k.cy))
      return set_err(ctx, GSR_ERR_INVALID_ARG, "non-finite camera");
  }
  if (!(o->eps2d >= 0.f)) return set_err(ctx, GSR_ERR_INVALID_ARG, "eps2d must be >= 0");
  return GSR_OK;
}

long long render_count(const gsr_gaussians* g) {
  if (!g->segs) return g->n;
  long long s = 0;
  for (int k = 0; k < g->nsegs; ++k) s += g->segs[k].count;
  return s;
}

CamBatch make_cams(const gsr_camera* cams, int C, long long* npix) {
  CamBatch cb;
  std::memset(&cb, 0, sizeof(cb));
  cb.C = C;
  int tiles = 0;
  long long pix = 0;
  for (int c = 0; c < C; ++c) {
    const gsr_camera& k = cams[c];
    DevCam& d = cb.cam[c];
    for (int i = 0; i < 3; ++i) {
      for (int j = 0; j < 3; ++j) d.R[i * 3 + j] = k.viewmat[i * 4 + j];
      d.t[i] = k.viewmat[i * 4 + 3];
    }
    d.fx = k.fx; d.fy = k.fy; d.cx = k.cx; d.cy = k.cy;
    d.limx = 1.3f * (0.5f * k.width) / k.fx;
    d.limy = 1.3f * (0.5f * k.height) / k.fy;
    d.znear = k.near_plane;
    d.zfar = k.far_plane;
    for (int j = 0; j < 3; ++j) {
      double s = 0;
      for (int i = 0; i < 3; ++i) s += static_cast<double>(k.viewmat[i * 4 + j]) * k.viewmat[i * 4 + 3];
      d.center[j] = static_cast<float>(-s);
    }
    d.W = k.width;
    d.H = k.height;
    d.tiles_x = (k.width + kTile - 1) / kTile;
    d.tiles_y = (k.height + kTile - 1) / kTile;
    d.tile_off = tiles;
    d.pix_off = pix;
    d.aff = k.appearance;
    tiles += d.tiles_x * d.tiles_y;
    pix += static_cast<long long>(k.width) * k.height;
  }
  cb.total_tiles = tiles;
  *npix = pix;
  return cb;
}


#define GSR_TRY_ALLOC(buf, bytes)                                          \
  do {                                                                     \
    if (!ensure(ctx, (buf), (bytes), s)) return set_err(ctx, GSR_ERR_OOM, "device allocation failed"); \
  } while (0)

struct BinOut {
  Buf* rec;
  Buf* owner;
  Buf* pvals_s;
  Buf* ranges;
};

// Preprocess + sort + bin into `bo`. Returns V and P through the pointers.
// Zeroes the spans on the side stream after the work queued on `s`; `done` marks the end.
// The fill is one small kernel (launch_zero_fill: a block per ctx->fill_blocks) rather than the
// runtime's memset, which occupies every SM and stalls the latency-bound stages it runs beside.
cudaError_t enqueue_fill(gsr_ctx* ctx, const FillSpans& f, cudaStream_t s, cudaEvent_t done) {
  cudaError_t e = cudaEventRecord(ctx->ev_fork, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0);
  if (e == cudaSuccess) {
    launch_zero_fill(f, ctx->fill_blocks, ctx->fill_gbs, ctx->side);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(done, ctx->side);
  return e;
}

size_t spans_total(const FillSpans& f) {
  size_t n = 0;
  for (int k = 0; k < f.count; ++k) n += f.len[k];
  return n;
}

// Floats [from, to) of the spans taken one after another.
FillSpans slice_spans(const FillSpans& f, size_t from, size_t to) {
  FillSpans out{};
  size_t base = 0;
  for (int k = 0; k < f.count; ++k) {
    const size_t lo = std::max(from, base), hi = std::min(to, base + f.len[k]);
    if (lo < hi) {
      out.ptr[out.count] = f.ptr[k] + (lo - base);
      out.len[out.count] = hi - lo;
      ++out.count;
    }
    base += f.len[k];
  }
  return out;
}

// The first part (ctx->fill_early of the bytes) of a requested gradient fill
// (gsr_param_grads_zero), queued after the work queued on `s` by a forward.
cudaError_t start_prezero_early(gsr_ctx* ctx, cudaStream_t s) {
  if (!ctx->prezero_requested || ctx->prezero_early || !(ctx->fill_early > 0.f)) return cudaSuccess;
  const size_t total = spans_total(ctx->prezero);
  const size_t to = std::min(total, static_cast<size_t>(static_cast<double>(total) * ctx->fill_early));
  if (to == 0) return cudaSuccess;
  const cudaError_t e = enqueue_fill(ctx, slice_spans(ctx->prezero, 0, to), s, ctx->ev_prezero_early);
  if (e == cudaSuccess) {
    ctx->prezero_early = true;
    ctx->prezero_queued = to;
  }
  return e;
}

// The rest of a requested gradient fill, queued after the work queued on `s`.
cudaError_t start_prezero(gsr_ctx* ctx, cudaStream_t s) {
  if (!ctx->prezero_requested) return cudaSuccess;
  ctx->prezero_requested = false;
  const size_t total = spans_total(ctx->prezero);
  cudaError_t e = cudaSuccess;
  if (ctx->prezero_queued < total) {
    e = enqueue_fill(ctx, slice_spans(ctx->prezero, ctx->prezero_queued, total), s, ctx->ev_prezero);
    ctx->prezero_pending = e == cudaSuccess;
  }
  ctx->prezero_queued = total;
  return e;
}

// Orders every queued part of a requested fill before the work queued on `s` next.
cudaError_t join_prezero(gsr_ctx* ctx, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (ctx->prezero_early) e = cudaStreamWaitEvent(s, ctx->ev_prezero_early, 0);
  if (e == cudaSuccess && ctx->prezero_pending) e = cudaStreamWaitEvent(s, ctx->ev_prezero, 0);
  return e;
}

void clear_prezero(gsr_ctx* ctx) {
  ctx->prezero_requested = ctx->prezero_pending = ctx->prezero_early = false;
  ctx->prezero_queued = 0;
}

// The per-Gaussian fields of GaussArgs (everything but the count and the segment map).
void set_gauss_fields(const gsr_gaussians* g, GaussArgs& ga) {
  ga.means = g->means;
  ga.scales = g->scales;
  ga.quats = g->quats;
  ga.opac = g->opacities;
  ga.sh = g->sh;
  ga.K = g->sh_coeffs;
  ga.deg = g->sh_degree;
  ga.attr_dtype = g->attr_dtype;
  ga.sh_dtype = g->sh_dtype;
  ga.quat_vec4 = g->attr_dtype == GSR_F32 && (reinterpret_cast<uintptr_t>(g->quats) % 16 == 0);
  ga.sh_vec4 = g->sh_dtype == GSR_F32 && (reinterpret_cast<uintptr_t>(g->sh) % 16 == 0) && ((3 * g->sh_coeffs) % 4 == 0);
  const bool eval = g->mlp && !g->mlp->cached;
  ga.gemb = eval ? g->mlp->gauss_embed : nullptr;
  ga.iemb = eval ? g->mlp->image_embed : nullptr;
  ga.mlp = eval ? g->mlp->params : nullptr;
  ga.mlp_cached = g->mlp ? g->mlp->cached : nullptr;
}

// Uploads the segment list (array index and selected index of each segment's first Gaussian, and
// the cameras that render it) and fills the kernels' segment map; an identity map without
// segments. Copies from pageable host memory return once the data is staged, so the host
// vectors may go when this returns and the stream is not synchronised.
gsr_status upload_segments(gsr_ctx* ctx, const gsr_gaussians* g, SegMap* m, cudaStream_t s) {
  m->nsegs = 0;
  m->begin = nullptr;
  m->start = nullptr;
  m->cams = nullptr;
  if (!g->segs) return GSR_OK;
  const int ns = std::max(g->nsegs, 1);
  GSR_TRY_ALLOC(ctx->seg_begin, sizeof(long long) * ns);
  GSR_TRY_ALLOC(ctx->seg_start, sizeof(long long) * ns);
  if (g->seg_cams) GSR_TRY_ALLOC(ctx->seg_cams, sizeof(uint32_t) * ns);
  std::vector<long long> hb(ns, 0), hs(ns, 0);
  std::vector<uint32_t> hc(ns, 0);
  long long acc = 0;
  for (int k = 0; k < g->nsegs; ++k) {
    hb[k] = g->segs[k].begin;
    hs[k] = acc;  // an empty segment starts where the next one does: the search takes the last
    acc += g->segs[k].count;
    if (g->seg_cams) hc[k] = g->seg_cams[k];
  }
  cudaError_t e = cudaMemcpyAsync(ctx->seg_begin.p, hb.data(), sizeof(long long) * ns, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ctx->seg_start.p, hs.data(), sizeof(long long) * ns, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && g->seg_cams)
    e = cudaMemcpyAsync(ctx->seg_cams.p, hc.data(), sizeof(uint32_t) * ns, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_err(ctx, e, "segment upload");
  m->nsegs = g->nsegs;
  m->begin = as<long long>(ctx->seg_begin);
  m->start = as<long long>(ctx->seg_start);
  m->cams = g->seg_cams ? as<uint32_t>(ctx->seg_cams) : nullptr;
  return GSR_OK;
}

// sort_in_blend: the per-tile lists of at most kTileSortSmall pairs are left unsorted in
// ctx->pair_keys for the forward blend to sort (only the longer lists are sorted here).
gsr_status run_binning(gsr_ctx* ctx, const gsr_gaussians* g, const CamBatch& cb, const gsr_opts* o, BinOut bo,
                       long long* V_out, long long* P_out, cudaStream_t s, long long* max_tile_out = nullptr,
                       bool sort_in_blend = false) {
  const long long N = render_count(g);
  const int C = cb.C;
  const long long capv = std::max<long long>(1, N * C);
  // segment map
  GaussArgs ga;
  ga.n_render = N;
  const gsr_status sst = upload_segments(ctx, g, &ga.segs, s);
  if (sst != GSR_OK) return sst;
  set_gauss_fields(g, ga);

  const int pre_blocks = static_cast<int>((N + kPreTile - 1) / kPreTile);
  const int tiles = cb.total_tiles;
  const bool global = o->global_sort != 0;
  GSR_TRY_ALLOC(*bo.rec, sizeof(Rec) * capv);
  GSR_TRY_ALLOC(*bo.owner, sizeof(uint32_t) * capv);
  GSR_TRY_ALLOC(*bo.ranges, sizeof(uint2) * std::max(tiles, 1));
  GSR_TRY_ALLOC(ctx->pre_vis, sizeof(uint32_t) * std::max<long long>(N, 1));
  GSR_TRY_ALLOC(ctx->pre_counts, sizeof(uint32_t) * std::max(pre_blocks, 1));
  const long long scan_items = global ? capv : tiles;
  const long long scan_blocks = (scan_items + kScanThreads * kScanItems - 1) / (kScanThreads * kScanItems);
  if (!ensure_zeroed(ctx, ctx->scan_status, sizeof(unsigned long long) * (scan_blocks + 1), s))
    return set_err(ctx, GSR_ERR_OOM, "device allocation failed");
  // misc (32-bit words): [0] unused, [1] V, [2] scan block counter,
  // [3] largest tile's pair count, [4..5] P (64-bit), [6] tiles listed for the large-list sort
  GSR_TRY_ALLOC(ctx->misc, 64);
  uint32_t* misc = as<uint32_t>(ctx->misc);
  uint32_t* d_V = misc + 1;
  unsigned long long* d_P = reinterpret_cast<unsigned long long*>(misc + 4);
  // The error word is not cleared here: a pair-placement overflow of the previous launch (which
  // runs after that launch's read-back) is reported by this one's, then the word is cleared.
  cudaError_t e = cudaMemsetAsync(ctx->misc.p, 0, 64, s);
  if (e != cudaSuccess) return cuda_err(ctx, e, "memset");

  PreOut po{};
  po.rec = as<Rec>(*bo.rec);
  po.owner = as<uint32_t>(*bo.owner);
  GSR_TRY_ALLOC(ctx->rcam, capv);
  po.rcam = as<uint8_t>(ctx->rcam);
  po.vis = as<uint32_t>(ctx->pre_vis);
  po.counts = as<uint32_t>(ctx->pre_counts);
  po.v_total = d_V;
  po.err = ctx->d_err;
  uint32_t* tile_ctr = nullptr;
  SortScratch sc{};
  if (global) {
    // depth keys of the records, sorted by the onesweep radix sort (the preprocess counts their digits)
    GSR_TRY_ALLOC(ctx->dkeys, sizeof(uint32_t) * capv);
    GSR_TRY_ALLOC(ctx->dvals, sizeof(uint32_t) * capv);
    GSR_TRY_ALLOC(ctx->touched, sizeof(uint32_t) * capv);
    GSR_TRY_ALLOC(ctx->dkeys_s, sizeof(uint32_t) * capv);
    GSR_TRY_ALLOC(ctx->dvals_s, sizeof(uint32_t) * capv);
    GSR_TRY_ALLOC(ctx->offsets, sizeof(uint32_t) * capv);
    if (!ensure_sort(ctx, capv, s)) return set_err(ctx, GSR_ERR_OOM, "device allocation failed");
    sc = sort_scratch(ctx);
    sort_clear_counts(sc, s);
    po.depth_keys = as<uint32_t>(ctx->dkeys);
    po.depth_vals = as<uint32_t>(ctx->dvals);
    po.touched = as<uint32_t>(ctx->touched);
    po.key_counts = sc.hist;
  } else {
    GSR_TRY_ALLOC(ctx->tile_ctr, sizeof(uint32_t) * std::max(tiles, 1));
    GSR_TRY_ALLOC(ctx->big_tiles, sizeof(uint32_t) * std::max(tiles, 1));
    tile_ctr = as<uint32_t>(ctx->tile_ctr);
    e = cudaMemsetAsync(tile_ctr, 0, sizeof(uint32_t) * tiles, s);
    if (e != cudaSuccess) return cuda_err(ctx, e, "memset");
    po.tile_ctr = tile_ctr;  // the record pass counts the pairs per tile
    po.tile_cull = o->tile_cull;
  }
  {
    StageTimer tm(ctx, GSR_STAGE_PREPROCESS, s);
    // the record pass: a grid of 8 blocks per SM (twice the resident ones; 16 per SM was measured
    // slower on the 6M city), never more than the records can use
    const int rec_blocks = static_cast<int>(std::min<long long>((capv + kPreThreads - 1) / kPreThreads,
                                                                 4LL * ctx->grid_cap));
    launch_preprocess_fwd(ga, cb, o->eps2d, o->antialiased, po, pre_blocks, rec_blocks, s);
  }
  e = start_prezero_early(ctx, s);
  if (e != cudaSuccess) return cuda_err(ctx, e, "gradient fill");
  if (global) {
    // records by depth, then (tile-culled) counts and pair offsets in depth order
    if (N * C > 0) {
      StageTimer tm(ctx, GSR_STAGE_DEPTH_SORT, s);
      radix_sort_u32(as<uint32_t>(ctx->dkeys), as<uint32_t>(ctx->dvals), as<uint32_t>(ctx->dkeys_s),
                     as<uint32_t>(ctx->dvals_s), d_V, capv, 0, 32, sc, next_epoch(ctx, s), false, true, ctx->d_err, s);
    }
    const uint32_t* cnt_sorted = nullptr;
    if (o->tile_cull && N * C > 0) {
      GSR_TRY_ALLOC(ctx->cnt_sorted, sizeof(uint32_t) * capv);
      StageTimer tm(ctx, GSR_STAGE_TILE_COUNT, s);
      launch_duplicate(as<Rec>(*bo.rec), as<uint32_t>(ctx->dvals_s), nullptr, d_V, capv, cb, 1,
                       as<uint32_t>(ctx->cnt_sorted), nullptr, nullptr, nullptr, 0, 4 * ctx->grid_cap, s);
      cnt_sorted = as<uint32_t>(ctx->cnt_sorted);
    }
    StageTimer tm(ctx, GSR_STAGE_TILE_SCAN, s);
    pair_offsets_scan(as<uint32_t>(ctx->touched), as<uint32_t>(ctx->dvals_s), cnt_sorted, as<uint32_t>(ctx->offsets),
                      d_V, capv, as<unsigned long long>(ctx->scan_status), misc + 2, d_P, ctx->d_err,
                      next_epoch(ctx, s), ctx->grid_cap, ctx->wait, s);
  } else {
    // each tile's range and the total P from the pairs per tile (counted by the record pass)
    StageTimer tm(ctx, GSR_STAGE_TILE_SCAN, s);
    launch_tile_scan(tile_ctr, as<uint2>(*bo.ranges), tiles, as<unsigned long long>(ctx->scan_status), misc + 2, d_P,
                     misc + 3, as<uint32_t>(ctx->big_tiles), misc + 6, next_epoch(ctx, s), ctx->d_err, ctx->wait,
                     ctx->grid_cap, s);
  }
  // read V, P, the largest tile and the error word
  uint32_t* h = static_cast<uint32_t*>(ctx->pinned);
  {
    StageTimer tm(ctx, GSR_STAGE_READBACK, s);
    e = cudaMemcpyAsync(h, misc, 32, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h + 8, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_err(ctx, e, "binning");
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(ctx, e, "binning launch");
  const long long V = N > 0 ? h[1] : 0;
  const uint32_t max_count = h[3];
  unsigned long long Pu;
  std::memcpy(&Pu, h + 4, sizeof(Pu));
  const int derr = static_cast<int>(h[8]);
  if (derr) {
    e = cudaMemsetAsync(ctx->d_err, 0, sizeof(int), s);
    if (e != cudaSuccess) return cuda_err(ctx, e, "memset");
  }
  if (derr & kErrTimeout) return set_err(ctx, GSR_ERR_DEVICE_TIMEOUT, "a bounded device wait ran out in binning");
  if (derr & kErrOverflow)
    return set_err(ctx, GSR_ERR_UNSUPPORTED, "pair count overflow (more than 2^32 pairs, or a placement past its tile)");
  if (V > capv) return set_err(ctx, GSR_ERR_CUDA, "inconsistent visible count");
  const long long P = V > 0 ? static_cast<long long>(Pu) : 0;
  if (P >= (1ll << 30)) return set_err(ctx, GSR_ERR_UNSUPPORTED, "more than 2^30 (tile, Gaussian) pairs");
  *V_out = V;
  *P_out = P;
  if (max_tile_out) *max_tile_out = P > 0 ? static_cast<long long>(max_count) : 0;

  const long long Pc = std::max<long long>(P, 1);
  GSR_TRY_ALLOC(*bo.pvals_s, sizeof(uint32_t) * Pc);
  if (global) {
    // pairs keyed by tile in depth order, sorted stably by tile, ranges by binary search
    GSR_TRY_ALLOC(ctx->pkeys, sizeof(uint32_t) * Pc);
    GSR_TRY_ALLOC(ctx->pvals, sizeof(uint32_t) * Pc);
    GSR_TRY_ALLOC(ctx->pkeys_s, sizeof(uint32_t) * Pc);
    if (P > 0) {
      if (!ensure_sort(ctx, Pc, s)) return set_err(ctx, GSR_ERR_OOM, "device allocation failed");
      sc = sort_scratch(ctx);
      int tb = 1;
      while ((1ll << tb) < tiles) ++tb;
      sort_clear_counts(sc, s);  // the pair emitter counts the tile keys' digits
      {
        StageTimer tm(ctx, GSR_STAGE_PLACE, s);
        launch_duplicate(as<Rec>(*bo.rec), as<uint32_t>(ctx->dvals_s), as<uint32_t>(ctx->offsets), d_V, V, cb,
                         o->tile_cull, nullptr, as<uint32_t>(ctx->pkeys), as<uint32_t>(ctx->pvals), sc.hist, tb,
                         4 * ctx->grid_cap, s);
      }
      {
        StageTimer tm(ctx, GSR_STAGE_TILE_SORT, s);
        radix_sort_u32(as<uint32_t>(ctx->pkeys), as<uint32_t>(ctx->pvals), as<uint32_t>(ctx->pkeys_s),
                       as<uint32_t>(*bo.pvals_s), nullptr, P, 0, tb, sc, next_epoch(ctx, s), false, true, ctx->d_err, s);
      }
    }
    StageTimer tm(ctx, GSR_STAGE_RANGES, s);
    if (P > 0) {
      launch_ranges(as<uint32_t>(ctx->pkeys_s), P, tiles, as<uint2>(*bo.ranges), s);
    } else {
      e = cudaMemsetAsync(bo.ranges->p, 0, sizeof(uint2) * std::max(tiles, 1), s);
      if (e != cudaSuccess) return cuda_err(ctx, e, "memset ranges");
    }
  } else if (P > 0) {
    // place the pairs in their tiles' ranges, then order every tile's list by (depth, index)
    GSR_TRY_ALLOC(ctx->pair_keys, sizeof(unsigned long long) * Pc);
    unsigned long long* scratch = nullptr;
    if (max_count > static_cast<uint32_t>(kTileSortCap)) {
      GSR_TRY_ALLOC(ctx->key_scratch, sizeof(unsigned long long) * Pc);
      scratch = as<unsigned long long>(ctx->key_scratch);
    }
    {
      StageTimer tm(ctx, GSR_STAGE_PLACE, s);
      launch_bin_pairs(as<Rec>(*bo.rec), d_V, V, cb, o->tile_cull, tile_ctr, as<uint2>(*bo.ranges),
                       as<unsigned long long>(ctx->pair_keys), ctx->d_err, 4 * ctx->grid_cap, s);
    }
    {
      StageTimer tm(ctx, GSR_STAGE_TILE_SORT, s);
      launch_tile_sort(as<unsigned long long>(ctx->pair_keys), as<uint2>(*bo.ranges), tiles, as<uint32_t>(*bo.pvals_s),
                       scratch, max_count, as<uint32_t>(ctx->big_tiles), misc + 6, !sort_in_blend, ctx->grid_cap, s);
    }
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(ctx, e, "pair launch");
  return GSR_OK;
}

}  // namespace

extern "C" {

const char* gsr_status_string(gsr_status s) {
  switch (s) {
    case GSR_OK: return "ok";
    case GSR_WARN_OVER_BUDGET: return "over budget";
    case GSR_ERR_INVALID_ARG: return "invalid argument";
    case GSR_ERR_OOM: return "out of device memory";
    case GSR_ERR_CUDA: return "CUDA error";
    case GSR_ERR_DEVICE_TIMEOUT: return "device wait timed out";
    case GSR_ERR_UNSUPPORTED: return "unsupported size";
  }
  return "unknown status";
}

gsr_status gsr_create(gsr_ctx** out, int device, const gsr_allocator* alloc) {
  if (!out) return GSR_ERR_INVALID_ARG;
  *out = nullptr;
  if (alloc && (!alloc->alloc || !alloc->free)) return GSR_ERR_INVALID_ARG;
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return GSR_ERR_CUDA;
  gsr_ctx* ctx = new (std::nothrow) gsr_ctx();
  if (!ctx) return GSR_ERR_OOM;
  ctx->device = device;
  if (alloc) {
    ctx->alloc = *alloc;
    ctx->has_alloc = true;
  }
  if (cudaMallocHost(&ctx->pinned, 256) != cudaSuccess || cudaMalloc(&ctx->d_err, 64) != cudaSuccess) {
    cudaGetLastError();
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    delete ctx;
    return GSR_ERR_OOM;
  }
  cudaMemset(ctx->d_err, 0, 64);
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) == cudaSuccess && sms > 0) {
    ctx->grid_cap = 2 * sms;
    ctx->fill_blocks = sms;
  }
  cudaGetLastError();
  if (!alloc) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    if (cudaMemPoolCreate(&ctx->pool, &props) == cudaSuccess) {
      unsigned long long keep = ~0ull;  // keep freed memory in the pool for reuse
      cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    } else {
      cudaGetLastError();
      ctx->pool = nullptr;  // fall back to cudaMalloc / cudaFree
    }
  }
  // the side stream carries the gradient fill; high priority lets its blocks take the SM room
  // the blend backward leaves instead of queueing behind that kernel's blocks
  int prio_least = 0, prio_greatest = 0;
  cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest);
  if (cudaStreamCreateWithPriority(&ctx->side, cudaStreamNonBlocking, prio_greatest) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_prezero, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_prezero_early, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    gsr_destroy(ctx);
    return GSR_ERR_CUDA;
  }
  *out = ctx;
  return GSR_OK;
}

void gsr_destroy(gsr_ctx* ctx) {
  if (!ctx) return;
  cudaDeviceSynchronize();
  for (gsr_fwd_state* st : ctx->state_pool) {
    Buf* sb[] = {&st->rec, &st->owner, &st->pvals_s, &st->ranges, &st->T_final, &st->n_contrib, &st->D};
    for (Buf* b : sb) release(ctx, *b, nullptr);
    delete st;
  }
  ctx->state_pool.clear();
  Buf* all[] = {&ctx->seg_begin, &ctx->seg_start, &ctx->seg_cams, &ctx->rec, &ctx->owner, &ctx->rcam, &ctx->sort_ktmp,
                &ctx->sort_vtmp, &ctx->sort_hist, &ctx->sort_status, &ctx->pre_vis, &ctx->pre_counts, &ctx->scan_status, &ctx->misc,
                &ctx->tile_ctr, &ctx->big_tiles, &ctx->pair_keys, &ctx->key_scratch, &ctx->pvals_s, &ctx->ranges, &ctx->pix_T,
                &ctx->pix_n, &ctx->pix_D, &ctx->g2d, &ctx->gaff, &ctx->dkeys, &ctx->dvals, &ctx->touched,
                &ctx->dkeys_s, &ctx->dvals_s, &ctx->offsets, &ctx->cnt_sorted, &ctx->pkeys, &ctx->pvals, &ctx->pkeys_s};
  for (Buf* b : all) release(ctx, *b, nullptr);
  for (auto& r : ctx->prof_recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (cudaEvent_t ev : ctx->ev_pool) cudaEventDestroy(ev);
  cudaDeviceSynchronize();
  if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  if (ctx->ev_prezero) cudaEventDestroy(ctx->ev_prezero);
  if (ctx->ev_prezero_early) cudaEventDestroy(ctx->ev_prezero_early);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  if (ctx->d_err) cudaFree(ctx->d_err);
  delete ctx;
}

const char* gsr_last_error(const gsr_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

size_t gsr_workspace_bytes(const gsr_ctx* ctx) { return ctx ? ctx->held : 0; }

gsr_status gsr_workspace_query(gsr_ctx* ctx, int64_t n_render, const gsr_camera* cams, int32_t n_cams,
                               int64_t expected_pairs, size_t* bytes_out) {
  if (!ctx || !cams || !bytes_out || n_cams < 1 || n_cams > kMaxCams || n_render < 0 || expected_pairs < 0)
    return GSR_ERR_INVALID_ARG;
  long long npix = 0;
  CamBatch cb = make_cams(cams, n_cams, &npix);
  const size_t capv = static_cast<size_t>(std::max<int64_t>(1, n_render * n_cams));
  const size_t P = static_cast<size_t>(std::max<int64_t>(1, expected_pairs));
  size_t b = 0;
  b += capv * (sizeof(Rec) + sizeof(uint32_t) + 1);              // records, owners, cameras
  b += static_cast<size_t>(n_render) * sizeof(uint32_t);         // visibility bits of the cull pass
  b += P * (2 * sizeof(unsigned long long) + sizeof(uint32_t));  // pair keys, merge scratch, sorted records
  b += static_cast<size_t>(cb.total_tiles) * (sizeof(uint2) + sizeof(uint32_t));  // ranges, counters
  b += static_cast<size_t>(npix) * 4 * sizeof(float);            // per-pixel state
  *bytes_out = b;
  return GSR_OK;
}

gsr_status gsr_render_forward(gsr_ctx* ctx, const gsr_gaussians* g, const gsr_camera* cams, int32_t n_cams,
                              const gsr_opts* opts, const gsr_outputs* out, gsr_fwd_state** state_out,
                              gsr_stream stream) {
  gsr_status st = validate(ctx, g, cams, n_cams, opts);
  if (st != GSR_OK) return st;
  if (!out || !out->rgb) return set_err(ctx, GSR_ERR_INVALID_ARG, "rgb output is required");
  if (state_out) *state_out = nullptr;
  ++ctx->call_seq;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_err(ctx, e, "cudaSetDevice");
  ctx->last_stream = s;
  long long npix = 0;
  const CamBatch cb = make_cams(cams, n_cams, &npix);
  const long long N = render_count(g);
  if (N * n_cams >= (1ll << 31)) return set_err(ctx, GSR_ERR_UNSUPPORTED, "more than 2^31 (camera, Gaussian) pairs");

  gsr_fwd_state* stt = nullptr;
  if (state_out) {
    if (!ctx->state_pool.empty()) {
      stt = ctx->state_pool.back();
      ctx->state_pool.pop_back();
    } else {
      stt = new (std::nothrow) gsr_fwd_state();
      if (!stt) return set_err(ctx, GSR_ERR_OOM, "host allocation failed");
    }
    stt->ctx = ctx;
    stt->info = gsr_state_info{};
    stt->has_bins = opts->save_state != 0;
  }
  BinOut bo;
  if (stt && stt->has_bins) {
    bo = BinOut{&stt->rec, &stt->owner, &stt->pvals_s, &stt->ranges};
  } else {
    bo = BinOut{&ctx->rec, &ctx->owner, &ctx->pvals_s, &ctx->ranges};
  }
  long long V = 0, P = 0, max_tile = 0;
  const bool sort_in_blend = opts->global_sort == 0;
  st = run_binning(ctx, g, cb, opts, bo, &V, &P, s, &max_tile, sort_in_blend);
  if (st != GSR_OK) {
    if (stt) gsr_state_release(ctx, stt);
    return st;
  }
  Buf* pT = stt ? &stt->T_final : &ctx->pix_T;
  Buf* pn = stt ? &stt->n_contrib : &ctx->pix_n;
  Buf* pD = stt ? &stt->D : &ctx->pix_D;
  if (!ensure(ctx, *pT, sizeof(float) * npix, s) || !ensure(ctx, *pn, sizeof(uint32_t) * npix, s) ||
      !ensure(ctx, *pD, sizeof(float2) * npix, s)) {
    if (stt) gsr_state_release(ctx, stt);
    return set_err(ctx, GSR_ERR_OOM, "device allocation failed");
  }
  BlendFwdOut bf;
  bf.rgb = out->rgb;
  bf.depth_acc = out->depth_acc;
  bf.depth_exp = out->depth_exp;
  bf.alpha = out->alpha;
  bf.T_final = as<float>(*pT);
  bf.n_contrib = as<uint32_t>(*pn);
  bf.D_state = as<float2>(*pD);
  {
    StageTimer tm(ctx, GSR_STAGE_BLEND_FWD, s);
    const unsigned long long* tile_keys = sort_in_blend && P > 0 ? as<unsigned long long>(ctx->pair_keys) : nullptr;
    launch_blend_fwd(as<Rec>(*bo.rec), as<uint32_t>(*bo.pvals_s), tile_keys, static_cast<uint32_t>(max_tile),
                     as<uint2>(*bo.ranges), cb, opts->bg, bf, counters_of(ctx), s);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    if (stt) gsr_state_release(ctx, stt);
    return cuda_err(ctx, e, "blend launch");
  }
  if (stt) {
    stt->info.n_render = N;
    stt->info.n_cams = n_cams;
    stt->info.n_visible = V;
    stt->info.n_pairs = P;
    stt->info.n_tiles = cb.total_tiles;
    stt->info.n_pixels = npix;
    stt->info.max_tile_pairs = max_tile;
    *state_out = stt;
  }
  return GSR_OK;
}

namespace {

FillSpans grad_spans(const gsr_gaussians* g, const gsr_param_grads* grads) {
  FillSpans f{};
  const size_t n = static_cast<size_t>(g->n);
  const auto add = [&f](float* p, size_t len) { f.ptr[f.count] = p; f.len[f.count] = len; ++f.count; };
  add(grads->means, 3 * n);
  add(grads->scales, 3 * n);
  add(grads->quats, 4 * n);
  add(grads->opacities, n);
  add(grads->sh, 3 * static_cast<size_t>(g->sh_coeffs) * n);
  if (grads->absgrad) add(grads->absgrad, 2 * n);
  if (g->mlp && grads->gauss_embed) add(grads->gauss_embed, static_cast<size_t>(kEmbG) * n);
  return f;
}

bool same_spans(const FillSpans& a, const FillSpans& b) {
  if (a.count != b.count) return false;
  for (int k = 0; k < a.count; ++k)
    if (a.ptr[k] != b.ptr[k] || a.len[k] != b.len[k]) return false;
  return true;
}

}  // namespace

gsr_status gsr_appearance_cache(gsr_ctx* ctx, const gsr_gaussians* g, int32_t image, float* out, gsr_stream stream) {
  if (!ctx) return GSR_ERR_INVALID_ARG;
  if (!g || !g->mlp || !out || image < 0 || g->n < 0)
    return set_err(ctx, GSR_ERR_INVALID_ARG, "null gaussians, transform or output, or a negative image row");
  const gsr_appearance_mlp* m = g->mlp;
  if (!m->image_embed || !m->params || (g->n > 0 && !m->gauss_embed))
    return set_err(ctx, GSR_ERR_INVALID_ARG, "null appearance-transform array");
  if (reinterpret_cast<uintptr_t>(out) % 16 != 0)
    return set_err(ctx, GSR_ERR_INVALID_ARG, "output must be 16-byte aligned");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_err(ctx, e, "cudaSetDevice");
  GaussArgs ga{};
  ga.gemb = m->gauss_embed;
  ga.iemb = m->image_embed + static_cast<size_t>(kEmbI) * image;
  ga.mlp = m->params;
  launch_mlp_cache(ga, g->n, out, 4 * ctx->grid_cap, reinterpret_cast<cudaStream_t>(stream));
  e = cudaGetLastError();
  return e == cudaSuccess ? GSR_OK : cuda_err(ctx, e, "appearance cache launch");
}

gsr_status gsr_param_grads_zero(gsr_ctx* ctx, const gsr_gaussians* g, const gsr_param_grads* grads,
                                gsr_stream stream) {
  if (!ctx) return GSR_ERR_INVALID_ARG;
  if (!g || !grads) return set_err(ctx, GSR_ERR_INVALID_ARG, "null gaussians or gradient struct");
  if (g->n < 0 || (g->n > 0 && g->sh_coeffs < 1)) return set_err(ctx, GSR_ERR_INVALID_ARG, "bad Gaussian count");
  if (g->n > 0 && (!grads->means || !grads->scales || !grads->quats || !grads->opacities || !grads->sh))
    return set_err(ctx, GSR_ERR_INVALID_ARG, "null parameter gradient array");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_err(ctx, e, "cudaSetDevice");
  // a fill queued for an earlier request still writes its arrays: order it before what follows
  e = join_prezero(ctx, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_err(ctx, e, "join");
  clear_prezero(ctx);
  if (g->n == 0) return GSR_OK;
  ctx->prezero = grad_spans(g, grads);
  ctx->prezero_requested = true;
  return GSR_OK;
}

gsr_status gsr_render_backward(gsr_ctx* ctx, const gsr_gaussians* g, const gsr_camera* cams, int32_t n_cams,
                               const gsr_opts* opts, const gsr_fwd_state* state, const gsr_out_grads* dout,
                               const gsr_param_grads* grads, gsr_stream stream) {
  gsr_status st = validate(ctx, g, cams, n_cams, opts);
  if (st != GSR_OK) return st;
  if (!state || state->ctx != ctx || !dout || !grads)
    return set_err(ctx, GSR_ERR_INVALID_ARG, "null state, upstream or gradient struct");
  if (g->n > 0 && (!grads->means || !grads->scales || !grads->quats || !grads->opacities || !grads->sh))
    return set_err(ctx, GSR_ERR_INVALID_ARG, "null parameter gradient array");
  if (g->mlp && g->mlp->cached)
    return set_err(ctx, GSR_ERR_UNSUPPORTED, "cached appearance outputs are for rendering only");
  if (g->mlp && (!grads->image_embed || !grads->mlp_params || (g->n > 0 && !grads->gauss_embed)))
    return set_err(ctx, GSR_ERR_INVALID_ARG, "null appearance-transform gradient array");
  const long long N = render_count(g);
  if (N != state->info.n_render || n_cams != state->info.n_cams)
    return set_err(ctx, GSR_ERR_INVALID_ARG, "inputs differ from the forward that made the state");
  ++ctx->call_seq;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_err(ctx, e, "cudaSetDevice");
  long long npix = 0;
  const CamBatch cb = make_cams(cams, n_cams, &npix);
  gsr_fwd_state* ms = const_cast<gsr_fwd_state*>(state);
  BinOut bo;
  long long V = state->info.n_visible;
  if (state->has_bins) {
    bo = BinOut{&ms->rec, &ms->owner, &ms->pvals_s, &ms->ranges};
  } else {
    bo = BinOut{&ctx->rec, &ctx->owner, &ctx->pvals_s, &ctx->ranges};
    long long P = 0;
    st = run_binning(ctx, g, cb, opts, bo, &V, &P, s);
    if (st != GSR_OK) return st;
    if (V != state->info.n_visible || P != state->info.n_pairs)
      return set_err(ctx, GSR_ERR_INVALID_ARG, "recomputed binning differs from the forward");
  }
  const long long Vc = std::max<long long>(V, 1);
  if (!ensure(ctx, ctx->g2d, sizeof(Grad2D) * Vc, s)) return set_err(ctx, GSR_ERR_OOM, "device allocation failed");
  e = cudaMemsetAsync(ctx->g2d.p, 0, sizeof(Grad2D) * Vc, s);
  if (e == cudaSuccess && grads->appearance)
    e = cudaMemsetAsync(grads->appearance, 0, sizeof(float) * 12 * n_cams, s);
  if (e == cudaSuccess && g->mlp) e = cudaMemsetAsync(grads->image_embed, 0, sizeof(float) * kEmbI * n_cams, s);
  if (e == cudaSuccess && g->mlp) e = cudaMemsetAsync(grads->mlp_params, 0, sizeof(float) * kMlpParams, s);
  if (e != cudaSuccess) return cuda_err(ctx, e, "memset");
  // Every parameter-gradient row starts at zero; only rows of Gaussians with a record are then
  // written. The fill is queued on the side stream right before the blend backward, which it
  // runs beside (measured against other placements: see gsr_set_fill_split); a share of a
  // requested fill that a forward already queued is waited for before the projection backward.
  bool join_requested = false;  // the projection backward waits for the requested fill
  cudaEvent_t join = nullptr;
  const bool requested = ctx->prezero_requested || ctx->prezero_pending || ctx->prezero_early;
  if (g->n > 0 && requested && same_spans(grad_spans(g, grads), ctx->prezero)) {
    e = start_prezero(ctx, s);  // what is left of it, beside the blend
    if (e != cudaSuccess) return cuda_err(ctx, e, "gradient fill");
    join_requested = true;
  } else {
    // arrays requested for zeroing other than these (or none to fill here): zero them too,
    // ordered before what follows
    e = start_prezero(ctx, s);
    if (e == cudaSuccess) e = join_prezero(ctx, s);
    if (e == cudaSuccess && g->n > 0) e = enqueue_fill(ctx, grad_spans(g, grads), s, ctx->ev_join);
    if (e != cudaSuccess) return cuda_err(ctx, e, "gradient fill");
    if (g->n > 0) join = ctx->ev_join;
    clear_prezero(ctx);
  }
  BlendBwdIn bi;
  bi.d_rgb = dout->rgb;
  bi.d_depth_acc = dout->depth_acc;
  bi.d_depth_exp = dout->depth_exp;
  bi.d_alpha = dout->alpha;
  bi.T_final = static_cast<const float*>(state->T_final.p);
  bi.n_contrib = static_cast<const uint32_t*>(state->n_contrib.p);
  bi.D_state = static_cast<const float2*>(state->D.p);
  {
    StageTimer tm(ctx, GSR_STAGE_BLEND_BWD, s);
    launch_blend_bwd(as<Rec>(*bo.rec), as<uint32_t>(*bo.pvals_s), as<uint2>(*bo.ranges), cb, opts->bg, bi,
                     as<Grad2D>(ctx->g2d), grads->appearance, opts->absgrad && grads->absgrad, counters_of(ctx), s);
  }
  if (join) e = cudaStreamWaitEvent(s, join, 0);
  if (e == cudaSuccess && join_requested) {
    e = join_prezero(ctx, s);
    clear_prezero(ctx);
  }
  if (e != cudaSuccess) return cuda_err(ctx, e, "join");
  GaussArgs ga;
  ga.n_render = N;
  // the segment table may have been overwritten by another call since the forward: upload it
  // again (the recompute path above has just done so)
  if (state->has_bins || !g->segs) {
    st = upload_segments(ctx, g, &ga.segs, s);
    if (st != GSR_OK) return st;
  } else {
    ga.segs.nsegs = g->nsegs;
    ga.segs.begin = as<long long>(ctx->seg_begin);
    ga.segs.start = as<long long>(ctx->seg_start);
    ga.segs.cams = g->seg_cams ? as<uint32_t>(ctx->seg_cams) : nullptr;
  }
  set_gauss_fields(g, ga);
  ParamGrads pg;
  pg.means = grads->means;
  pg.scales = grads->scales;
  pg.quats = grads->quats;
  pg.opac = grads->opacities;
  pg.sh = grads->sh;
  pg.absgrad = opts->absgrad ? grads->absgrad : nullptr;
  pg.vec4 = (reinterpret_cast<uintptr_t>(grads->quats) % 16 == 0) && (reinterpret_cast<uintptr_t>(grads->sh) % 16 == 0) &&
            ((3 * g->sh_coeffs) % 4 == 0);
  if (g->mlp) {
    // the appearance transform's backward turns the records' gradients into those of the
    // transform's inputs before the projection backward reads them
    StageTimer tm(ctx, GSR_STAGE_APPEARANCE_BWD, s);
    launch_mlp_bwd(ga, cb, V, as<Rec>(*bo.rec), as<uint32_t>(*bo.owner), as<Grad2D>(ctx->g2d), grads->gauss_embed,
                   grads->image_embed, grads->mlp_params, 3 * (ctx->grid_cap / 2), s);
  }
  {
    StageTimer tm(ctx, GSR_STAGE_PREPROCESS_BWD, s);
    launch_preprocess_bwd(ga, cb, opts->eps2d, opts->antialiased, V, as<Rec>(*bo.rec), as<uint32_t>(*bo.owner),
                          as<Grad2D>(ctx->g2d), pg, s);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_err(ctx, e, "backward launch");
  return GSR_OK;
}

void gsr_state_release(gsr_ctx* ctx, gsr_fwd_state* state) {
  if (!state) return;
  gsr_ctx* c = ctx ? ctx : state->ctx;
  // Keep up to a few released states with their buffers: the next forward on this context's
  // stream reuses them in stream order, without a cudaFree or a device synchronisation.
  constexpr size_t kPoolMax = 4;
  if (c && c->state_pool.size() < kPoolMax) {
    c->state_pool.push_back(state);
    return;
  }
  Buf* all[] = {&state->rec, &state->owner, &state->pvals_s, &state->ranges, &state->T_final, &state->n_contrib,
                &state->D};
  if (c)
    for (Buf* b : all) release(c, *b, c->last_stream);
  delete state;
}

gsr_status gsr_state_get_info(const gsr_fwd_state* state, gsr_state_info* info) {
  if (!state || !info) return GSR_ERR_INVALID_ARG;
  *info = state->info;
  return GSR_OK;
}

gsr_status gsr_state_copy(const gsr_fwd_state* state, int32_t which, void* dst, size_t bytes, gsr_stream stream) {
  if (!state || !dst) return GSR_ERR_INVALID_ARG;
  const gsr_ctx* ctx = state->ctx;
  const void* src = nullptr;
  size_t have = 0;
  auto pick = [&](const Buf& own, const Buf& scratch, size_t n) {
    const Buf& b = state->has_bins ? own : scratch;
    src = b.p;
    have = std::min(n, b.cap);
  };
  const gsr_state_info& I = state->info;
  switch (which) {
    case GSR_BUF_RECORDS: pick(state->rec, ctx->rec, sizeof(Rec) * I.n_visible); break;
    case GSR_BUF_OWNER: pick(state->owner, ctx->owner, 4 * I.n_visible); break;
    case GSR_BUF_PAIR_VALS: pick(state->pvals_s, ctx->pvals_s, 4 * I.n_pairs); break;
    case GSR_BUF_RANGES: pick(state->ranges, ctx->ranges, 8 * I.n_tiles); break;
    case GSR_BUF_T_FINAL: src = state->T_final.p; have = std::min<size_t>(4 * I.n_pixels, state->T_final.cap); break;
    case GSR_BUF_N_CONTRIB: src = state->n_contrib.p; have = std::min<size_t>(4 * I.n_pixels, state->n_contrib.cap); break;
    case GSR_BUF_DEPTH_STATE: src = state->D.p; have = std::min<size_t>(8 * I.n_pixels, state->D.cap); break;
    default: return GSR_ERR_INVALID_ARG;
  }
  if (!src || bytes > have) return GSR_ERR_INVALID_ARG;
  if (bytes == 0) return GSR_OK;
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? GSR_OK : GSR_ERR_CUDA;
}

gsr_status gsr_sync_check(gsr_ctx* ctx, gsr_stream stream) {
  if (!ctx) return GSR_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_err(ctx, e, "sync");
  if (h) {
    cudaMemsetAsync(ctx->d_err, 0, sizeof(int), s);
    if (h & kErrTimeout) return set_err(ctx, GSR_ERR_DEVICE_TIMEOUT, "a bounded device wait ran out");
    return set_err(ctx, GSR_ERR_UNSUPPORTED, "a device count overflowed");
  }
  return GSR_OK;
}

gsr_status gsr_set_fill_rate(gsr_ctx* ctx, float gb_per_s, int32_t blocks) {
  if (!ctx || !(gb_per_s >= 0.f) || blocks < 0) return GSR_ERR_INVALID_ARG;
  ctx->fill_gbs = gb_per_s;
  if (blocks > 0) ctx->fill_blocks = blocks;
  return GSR_OK;
}

gsr_status gsr_set_fill_split(gsr_ctx* ctx, float early_share) {
  if (!ctx || !(early_share >= 0.f && early_share <= 1.f)) return GSR_ERR_INVALID_ARG;
  ctx->fill_early = early_share;
  return GSR_OK;
}

gsr_status gsr_set_wait_limit(gsr_ctx* ctx, uint32_t polls, int32_t never_ready) {
  if (!ctx) return GSR_ERR_INVALID_ARG;
  ctx->wait.limit = polls ? polls : kSpinLimit;
  ctx->wait.never_ready = never_ready ? 1u : 0u;
  return GSR_OK;
}

gsr_status gsr_profile_enable(gsr_ctx* ctx, int32_t on, int32_t count_evals) {
  if (!ctx) return GSR_ERR_INVALID_ARG;
  ctx->prof = on != 0;
  ctx->count_evals = count_evals != 0;
  return GSR_OK;
}

gsr_status gsr_profile_select(gsr_ctx* ctx, uint32_t stage_mask) {
  if (!ctx) return GSR_ERR_INVALID_ARG;
  ctx->prof_mask = stage_mask;
  return GSR_OK;
}

gsr_status gsr_profile_collect(gsr_ctx* ctx, double* ms, int64_t* launches, int64_t* counters) {
  if (!ctx) return GSR_ERR_INVALID_ARG;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_err(ctx, e, "cudaSetDevice");
  const gsr_ctx::Rec3* prev = nullptr;
  for (auto& r : ctx->prof_recs) {
    float t = 0.f, gap = 0.f;
    const bool same_call = prev && prev->call == r.call;
    e = cudaEventSynchronize(r.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
    if (e == cudaSuccess && same_call) e = cudaEventElapsedTime(&gap, prev->b, r.a);
    if (e != cudaSuccess) return cuda_err(ctx, e, "profile events");
    if (ms) {
      ms[r.stage] += t;
      // time between the end of one stage and the start of the next within one call: memsets,
      // waits on the side stream or the host, launch latency
      if (same_call && gap > 0.f) ms[GSR_STAGE_BETWEEN] += gap;
    }
    if (launches) launches[r.stage] += 1;
    prev = &r;
  }
  for (auto& r : ctx->prof_recs) {
    ctx->ev_pool.push_back(r.a);
    ctx->ev_pool.push_back(r.b);
  }
  ctx->prof_recs.clear();
  unsigned long long h[GSR_NUM_COUNTERS] = {};
  e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(h, reinterpret_cast<char*>(ctx->d_err) + 8, sizeof(h), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(reinterpret_cast<char*>(ctx->d_err) + 8, 0, sizeof(h));
  if (e != cudaSuccess) return cuda_err(ctx, e, "profile counters");
  if (counters)
    for (int k = 0; k < GSR_NUM_COUNTERS; ++k) counters[k] += static_cast<int64_t>(h[k]);
  return GSR_OK;
}

gsr_status gsr_sort_pairs_u32(gsr_ctx* ctx, const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                              uint32_t* vals_out, int64_t n, int32_t begin_bit, int32_t end_bit, gsr_stream stream) {
  if (!ctx) return GSR_ERR_INVALID_ARG;
  if (n < 0 || begin_bit < 0 || end_bit > 32 || end_bit < begin_bit)
    return set_err(ctx, GSR_ERR_INVALID_ARG, "bad size or bit range");
  if (n > 0 && (!keys_in || !vals_in || !keys_out || !vals_out))
    return set_err(ctx, GSR_ERR_INVALID_ARG, "null pointer");
  if (n >= (1ll << 30)) return set_err(ctx, GSR_ERR_UNSUPPORTED, "n must be below 2^30");
  if (n == 0) return GSR_OK;
  if (keys_out == keys_in || vals_out == vals_in) return set_err(ctx, GSR_ERR_INVALID_ARG, "outputs alias inputs");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_err(ctx, e, "cudaSetDevice");
  if (end_bit == begin_bit) {
    e = cudaMemcpyAsync(keys_out, keys_in, 4 * n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(vals_out, vals_in, 4 * n, cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? GSR_OK : cuda_err(ctx, e, "copy");
  }
  if (!ensure_sort(ctx, n, s)) return set_err(ctx, GSR_ERR_OOM, "device allocation failed");
  SortScratch sc = sort_scratch(ctx);
  radix_sort_u32(keys_in, vals_in, keys_out, vals_out, nullptr, n, begin_bit, end_bit, sc, next_epoch(ctx, s), false,
                 false, ctx->d_err, s);
  e = cudaGetLastError();
  return e == cudaSuccess ? GSR_OK : cuda_err(ctx, e, "sort launch");
}

gsr_status gsr_select_lod(int32_t P, const double* aabb, int32_t L, const int64_t* level_offsets,
                          const gsr_camera* cam, const double* thresholds, int64_t budget, int32_t* levels,
                          gsr_segment* segs, int32_t* nsegs, int64_t* n_selected) {
  if (P < 0 || L < 1 || !cam || !levels || !nsegs || !n_selected || (P > 0 && (!aabb || !level_offsets || !segs)) ||
      (L > 1 && !thresholds))
    return GSR_ERR_INVALID_ARG;
  for (int k = 0; k + 1 < L - 1; ++k)
    if (!(thresholds[k] <= thresholds[k + 1])) return GSR_ERR_INVALID_ARG;
  // camera in double precision
  double R[9], t[3], ctr[3];
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) R[i * 3 + j] = cam->viewmat[i * 4 + j];
    t[i] = cam->viewmat[i * 4 + 3];
  }
  for (int j = 0; j < 3; ++j) ctr[j] = -(R[0 * 3 + j] * t[0] + R[1 * 3 + j] * t[1] + R[2 * 3 + j] * t[2]);
  const double fx = cam->fx, fy = cam->fy, cx = cam->cx, cy = cam->cy, W = cam->width, H = cam->height;
  const double zn = cam->near_plane, zf = cam->far_plane;
  std::vector<double> dist(P, 0.0);
  std::vector<int> lev(P, -1);
  int64_t total = 0;
  for (int p = 0; p < P; ++p) {
    const double* b = aabb + 6 * p;
    // corner k in camera space; culled iff all corners violate one half-space
    unsigned out_all = 0x3f;
    for (int k = 0; k < 8; ++k) {
      const double wx = (k & 1) ? b[3] : b[0], wy = (k & 2) ? b[4] : b[1], wz = (k & 4) ? b[5] : b[2];
      const double x = R[0] * wx + R[1] * wy + R[2] * wz + t[0];
      const double y = R[3] * wx + R[4] * wy + R[5] * wz + t[1];
      const double z = R[6] * wx + R[7] * wy + R[8] * wz + t[2];
      unsigned o = 0;
      if (z < zn) o |= 1;
      if (z > zf) o |= 2;
      if (fx * x + cx * z < 0.0) o |= 4;
      if (fx * x + (cx - W) * z > 0.0) o |= 8;
      if (fy * y + cy * z < 0.0) o |= 16;
      if (fy * y + (cy - H) * z > 0.0) o |= 32;
      out_all &= o;
    }
    double d2 = 0.0;
    for (int k = 0; k < 3; ++k) {
      const double q = std::min(std::max(ctr[k], b[k]), b[3 + k]);
      d2 += (ctr[k] - q) * (ctr[k] - q);
    }
    dist[p] = std::sqrt(d2);
    if (out_all) continue;
    int l = 0;
    for (int k = 0; k < L - 1; ++k)
      if (dist[p] < thresholds[k]) {
        l = L - 1 - k;
        break;
      }
    lev[p] = l;
  }
  auto cnt = [&](int p, int l) {
    return level_offsets[static_cast<int64_t>(l) * (P + 1) + p + 1] - level_offsets[static_cast<int64_t>(l) * (P + 1) + p];
  };
  for (int p = 0; p < P; ++p)
    if (lev[p] >= 0) total += cnt(p, lev[p]);
  gsr_status status = GSR_OK;
  if (budget > 0 && total > budget) {
    // farthest first: order candidates once by (distance desc, index desc)
    std::vector<int> order;
    for (int p = 0; p < P; ++p)
      if (lev[p] > 0) order.push_back(p);
    std::sort(order.begin(), order.end(), [&](int a, int b) {
      if (dist[a] != dist[b]) return dist[a] > dist[b];
      return a > b;
    });
    for (int p : order) {
      while (lev[p] > 0 && total > budget) {
        total -= cnt(p, lev[p]);
        lev[p] -= 1;
        total += cnt(p, lev[p]);
      }
      if (total <= budget) break;
    }
    if (total > budget) status = GSR_WARN_OVER_BUDGET;
  }
  int ns = 0;
  for (int p = 0; p < P; ++p) {
    levels[p] = lev[p];
    if (lev[p] < 0) continue;
    const int64_t c = cnt(p, lev[p]);
    if (c <= 0) continue;
    segs[ns].begin = level_offsets[static_cast<int64_t>(lev[p]) * (P + 1) + p];
    segs[ns].count = c;
    ++ns;
  }
  *nsegs = ns;
  *n_selected = total;
  return status;
}

}  // extern "C"
