// Internal declarations shared by the CUDA translation units of libgsr (sm_103a).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace gsr {

constexpr int kTile = 16;           // tile edge in pixels
constexpr int kTilePix = kTile * kTile;
constexpr int kMaxCams = 32;        // cameras per launch (bit mask of visibility is 32 bits)
constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kTMin = 1e-4f;

// Device error bits (ctx error word).
constexpr int kErrTimeout = 1;      // a chained-scan look-back gave up
constexpr int kErrOverflow = 2;     // a count did not fit the buffer it was sized for

// Bound on the polls of one look-back step before it reports kErrTimeout (with a nanosleep of
// up to 1 us between polls this is well under a second).
constexpr unsigned kSpinLimit = 1u << 20;

// How the chained-scan look-backs wait: `limit` polls per step before giving up (kErrTimeout),
// and `never_ready` (a test switch) makes every look-back treat its predecessors' status words as
// unpublished, so that each wait runs to the limit. A wait that gives up uses the partial prefix
// it has summed, which is never larger than the true one, so every write stays in bounds.
struct WaitCfg {
  unsigned limit = kSpinLimit;
  unsigned never_ready = 0;
};

struct DevCam {
  float R[9];
  float t[3];
  float fx, fy, cx, cy;
  float limx, limy;       // Jacobian clamp of X/Z and Y/Z
  float znear, zfar;
  float center[3];        // camera centre in world coordinates
  int W, H, tiles_x, tiles_y;
  int tile_off;           // first global tile index of this camera
  long long pix_off;      // first packed pixel of this camera
  const float* aff;       // [3,4] appearance transform or nullptr
};

struct CamBatch {
  int C;
  int total_tiles;
  DevCam cam[kMaxCams];
};

// Selected-index -> array-index map for segment lists.
struct SegMap {
  int nsegs;                   // 0: identity
  const long long* begin;      // [nsegs] array index of the segment's first Gaussian
  const long long* start;      // [nsegs] selected index of the segment's first Gaussian
  const uint32_t* cams;        // [nsegs] cameras of the launch that render the segment, or NULL (all)
};

// Splat record: 64 bytes (two 32-byte sectors), read by the blend kernels through the sorted
// pair list.
//   a = (mean2d x, mean2d y, opacity', view depth z)
//   b = (conic a, conic b, conic c, red)
//   c = (green, blue, bits(x0 | x1 << 16), bits(y0 | y1 << 16 | camera << 27))
//   d = (x min, x max, y min, y max) of the region where alpha can reach 1/255, slightly widened:
//       the blend kernels skip a Gaussian for a whole warp whose pixels all lie outside it.
struct __align__(16) Rec {
  float4 a, b, c, d;
};
__device__ __forceinline__ int rec_cam(const Rec& r) { return static_cast<int>(__float_as_uint(r.c.w) >> 27); }

template <typename T>
__device__ __forceinline__ float ldf(const T* p, long long i);
template <>
__device__ __forceinline__ float ldf<float>(const float* p, long long i) { return __ldg(p + i); }
template <>
__device__ __forceinline__ float ldf<__half>(const __half* p, long long i) { return __half2float(p[i]); }
template <>
__device__ __forceinline__ float ldf<__nv_bfloat16>(const __nv_bfloat16* p, long long i) {
  return __bfloat162float(p[i]);
}

__device__ __forceinline__ int seg_of(const SegMap& m, long long i) {
  int lo = 0, hi = m.nsegs - 1;
  while (lo < hi) {  // last segment with start <= i
    int mid = (lo + hi + 1) >> 1;
    if (m.start[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ long long seg_map(const SegMap& m, long long i) {
  if (m.nsegs == 0) return i;
  const int k = seg_of(m, i);
  return m.begin[k] + (i - m.start[k]);
}

// seg_map, and the cameras of the launch that render selected Gaussian i (bit c = camera c).
__device__ __forceinline__ long long seg_map_cams(const SegMap& m, long long i, uint32_t* cams) {
  if (m.nsegs == 0) {
    *cams = 0xffffffffu;
    return i;
  }
  const int k = seg_of(m, i);
  *cams = m.cams ? m.cams[k] : 0xffffffffu;
  return m.begin[k] + (i - m.start[k]);
}

// ---- arguments of the kernels ---------------------------------------------------------------

struct GaussArgs {
  long long n_render;  // Gaussians rendered
  SegMap segs;
  const float* means;
  const void* scales;
  const void* quats;
  const void* opac;
  const void* sh;
  int K;               // stored SH coefficients
  int deg;
  int attr_dtype;
  int sh_dtype;
  int quat_vec4;       // float32 quaternions on a 16-byte boundary: load each as one float4
  int sh_vec4;         // float32 SH rows on 16-byte boundaries (3K % 4 == 0): load as float4
  // appearance transform (gsr_appearance_mlp), all NULL when off
  const float* gemb;   // [n][16]
  const float* iemb;   // [C][32]
  const float* mlp;    // [kMlpParams]
  const float* mlp_cached;  // [n][4] outputs for one image embedding (rendering), or NULL
};

// Appearance transform sizes (the paper's): l_G 16, l_I 32, hidden 32, outputs 4.
constexpr int kEmbG = 16, kEmbI = 32, kHid = 32, kMlpOut = 4;
constexpr int kMlpIn = kEmbG + kEmbI;
constexpr int kMlpB1 = kHid * kMlpIn;           // offset of b1 in the packed parameters
constexpr int kMlpW2 = kMlpB1 + kHid;           // offset of w2
constexpr int kMlpB2 = kMlpW2 + kMlpOut * kHid; // offset of b2
constexpr int kMlpParams = kMlpB2 + kMlpOut;    // 1700

struct PreOut {
  Rec* rec;                    // [cap_v]
  uint32_t* owner;             // [cap_v] rendered index of the Gaussian of each record
  uint8_t* rcam;               // [cap_v] camera of each record (between the passes)
  uint32_t* vis;               // [n_render] camera bits of each Gaussian's visible records
  uint32_t* counts;            // [blocks] records per cull block, then each block's first record
  // the global-sort binning only (null otherwise): depth keys and record indices for the depth
  // sort, tiles in each record's rectangle, and the keys' digit counts [4][256] (added to)
  uint32_t* depth_keys;
  uint32_t* depth_vals;
  uint32_t* touched;
  uint32_t* key_counts;
  // the per-tile binning only (null otherwise): per-tile pair counts, added to (zeroed before),
  // with or without the StopThePop tile cull
  uint32_t* tile_ctr;
  int tile_cull;
  uint32_t* v_total;           // out: V
  int* err;
};

struct Grad2D {  // per visible record: 12 floats, three float4
  float4 a;      // mean2d x, mean2d y, opacity', depth
  float4 b;      // conic a, conic b, conic c, red
  float4 c;      // green, blue, |mean2d x|, |mean2d y|
};

struct ParamGrads {
  float* means;
  float* scales;
  float* quats;
  float* opac;
  float* sh;
  float* absgrad;
  int vec4;  // quats and SH rows may be stored as float4 (16-byte aligned, 3K % 4 == 0)
};

// ---- host-side launchers (one per translation unit) -------------------------------------

// The forward preprocess: the cull pass over all Gaussians (`blocks` blocks of kPreTile), the
// scan of its block counts, the compaction of the records' (Gaussian, camera), then the record
// pass over the visible records (`rec_blocks` blocks, grid-stride).
void launch_preprocess_fwd(const GaussArgs& g, const CamBatch& cams, float eps2d, int antialiased,
                           const PreOut& out, int blocks, int rec_blocks, cudaStream_t s);
void launch_preprocess_rec(const GaussArgs& g, const CamBatch& cams, float eps2d, int antialiased,
                           const PreOut& out, int rec_blocks, cudaStream_t s);
constexpr int kFillSpans = 8;
struct FillSpans {
  float* ptr[kFillSpans];
  size_t len[kFillSpans];  // floats
  int count;
};
// Sets `count` float arrays to zero with `blocks` blocks, at about gb_per_s (0: unpaced).
void launch_zero_fill(const FillSpans& f, int blocks, float gb_per_s, cudaStream_t s);
// Backward of the appearance transform, one thread per visible record (before
// launch_preprocess_bwd): turns the record's gradients of the transformed opacity and colour into
// those of the untransformed ones (in place in g2d), adds l_G's gradient to g_gemb (atomics; rows
// zeroed before) and sums the gradients of the weights and image embeddings into g_params and
// g_iemb (atomics; zeroed before).
// The appearance transform of Gaussians [0, n) for the image embedding at A.iemb into out.
void launch_mlp_cache(const GaussArgs& A, long long n, float* out, int blocks, cudaStream_t s);
void launch_mlp_bwd(const GaussArgs& g, const CamBatch& cams, long long V, const Rec* rec, const uint32_t* owner,
                    Grad2D* g2d, float* g_gemb, float* g_iemb, float* g_params, int blocks, cudaStream_t s);
// Runs over the V visible records; the first record of each Gaussian writes its gradient rows
// (the rows of Gaussians with no record must already be zero).
void launch_preprocess_bwd(const GaussArgs& g, const CamBatch& cams, float eps2d, int antialiased, long long V,
                           const Rec* rec, const uint32_t* owner, const Grad2D* g2d, const ParamGrads& out,
                           cudaStream_t s);
constexpr int kPreThreads = 256;
constexpr int kPreItems = 4;
constexpr int kPreTile = kPreThreads * kPreItems;

// Stable radix sort by key bits [begin_bit, end_bit); n taken from *d_n when d_n != nullptr
// (then max_n bounds it and sizes the launch), else n = max_n.
// Digit counts [4][256] followed by the four passes' block counters: zeroed together before
// the keys' digits are counted.
constexpr int kSortCountWords = 4 * 256 + 4;
struct SortScratch {
  uint32_t* keys_tmp;
  uint32_t* vals_tmp;
  uint32_t* hist;                // [kSortCountWords]: digit counts per pass, then block counters
  unsigned long long* status;    // [4][tiles][256] epoch-tagged look-back words
  int grid_cap;                  // blocks per onesweep launch (resident blocks loop over tiles)
  WaitCfg wait;
};
// Adds key's digits of passes [0, passes) (8 bits each from begin_bit, the last one up to
// end_bit) to a block's shared counts sh[4][256].
__device__ __forceinline__ void count_digits(uint32_t key, int begin_bit, int end_bit, int passes, uint32_t* sh) {
  for (int p = 0; p < passes; ++p) {
    const int shift = begin_bit + 8 * p;
    const int width = end_bit - shift < 8 ? end_bit - shift : 8;
    atomicAdd(&sh[p * 256 + ((key >> shift) & ((1u << width) - 1))], 1u);
  }
}
// Adds a block's nonzero shared counts to the global counts (whole block; the caller syncs
// before).
__device__ __forceinline__ void flush_digit_counts(const uint32_t* sh, int passes, uint32_t* hist) {
  for (int k = threadIdx.x; k < passes * 256; k += blockDim.x)
    if (sh[k]) atomicAdd(hist + k, sh[k]);
}
void sort_clear_counts(const SortScratch& sc, cudaStream_t s);
constexpr int kSortThreads = 512;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;
size_t sort_status_words(long long max_n);  // 64-bit words per pass
// epoch: tag for this call's status words (nonzero, below 2^30); clear_status: zero the status
// words first instead of relying on the tag; counts_ready: sc.hist already holds the keys' digit
// counts (sort_clear_counts, then count_digits / flush_digit_counts in the producing kernel).
void radix_sort_u32(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out, uint32_t* vals_out,
                    const uint32_t* d_n, long long max_n, int begin_bit, int end_bit, const SortScratch& sc,
                    uint32_t epoch, bool clear_status, bool counts_ready, int* err, cudaStream_t s);

// Binning of the V visible records (V read from *d_n, at most max_n) into (tile, record) pairs,
// once the preprocess's record pass has added each tile's pair count to tile_ctr (PreOut):
// launch_tile_scan turns the counts into ranges [start, end), P (*p_total), the largest count
// (*max_count, zeroed before), the list of tiles with more than kTileSortSmall pairs (big,
// *n_big zeroed before) and per-tile cursors (in tile_ctr); launch_bin_pairs places each pair's
// key (depth bits << 32 | record) in its tile's range (a pair past the range end sets
// kErrOverflow in *err and is not written); launch_tile_sort sorts every tile's keys (with
// small = false only the listed tiles of more than kTileSortSmall pairs: the forward blend sorts
// the others) and writes the records in that order into vals. Tiles with more than
// kTileSortCap pairs are sorted in runs merged through `scratch` ([P], null when max_count is
// at most kTileSortCap).
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kTileSortSmall = 1024;  // tiles up to this many pairs: one small block each
constexpr int kTileSortCap = 16384;   // keys a large block sorts in shared memory (128 KB)
void launch_bin_pairs(const Rec* rec, const uint32_t* d_n, long long max_n, const CamBatch& cams, int tile_cull,
                      uint32_t* tile_ctr, const uint2* ranges, unsigned long long* keys, int* err, int max_blocks,
                      cudaStream_t s);
void launch_tile_scan(uint32_t* tile_ctr, uint2* ranges, int n_tiles, unsigned long long* status, uint32_t* counter,
                      unsigned long long* p_total, uint32_t* max_count, uint32_t* big, uint32_t* n_big, uint32_t epoch,
                      int* err, WaitCfg wait, int grid_cap, cudaStream_t s);
void launch_tile_sort(unsigned long long* keys, const uint2* ranges, int n_tiles, uint32_t* vals,
                      unsigned long long* scratch, uint32_t max_count, const uint32_t* big, const uint32_t* n_big,
                      bool small, int grid_cap, cudaStream_t s);

// The global-sort binning (gsr_opts.global_sort). pair_offsets_scan: exclusive scan of per-record
// tile counts in depth order (counts[i] = touched[order[i]], or cnt_sorted[i] when given) into
// offsets, *p_total = P, n from *d_n. launch_duplicate: with cnt_sorted, the tile-culled count of
// each record in depth order; else the (tile id, record) pairs at the records' offsets (counting
// the tile keys' digits for their sort). launch_ranges: each tile's [start, end) in the sorted keys.
void pair_offsets_scan(const uint32_t* touched, const uint32_t* order, const uint32_t* cnt_sorted,
                       uint32_t* offsets, const uint32_t* d_n, long long max_n, unsigned long long* status,
                       uint32_t* counter, unsigned long long* p_total, int* err, uint32_t epoch, int grid_cap,
                       WaitCfg wait, cudaStream_t s);
void launch_duplicate(const Rec* rec, const uint32_t* order, const uint32_t* offsets, const uint32_t* d_n,
                      long long max_n, const CamBatch& cams, int tile_cull, uint32_t* cnt_sorted,
                      uint32_t* pair_keys, uint32_t* pair_vals, uint32_t* key_counts, int key_bits, int max_blocks,
                      cudaStream_t s);
void launch_ranges(const uint32_t* sorted_keys, long long P, int n_tiles, uint2* ranges, cudaStream_t s);

struct BlendFwdOut {
  float* rgb;
  float* depth_acc;
  float* depth_exp;
  float* alpha;
  float* T_final;
  uint32_t* n_contrib;
  float2* D_state;  // per pixel: depth of the first contributor, sum of (z - that depth) w
};
// counters (nullable): [0] evaluations, [1] contributions (forward), [2], [3] (backward)
// tile_keys (nullable): sort the lists of at most kTileSortSmall pairs in the blend from these
// unsorted keys (max_count: the longest list) and write their record order to pair_vals.
void launch_blend_fwd(const Rec* rec, uint32_t* pair_vals, const unsigned long long* tile_keys, uint32_t max_count,
                      const uint2* ranges, const CamBatch& cams, const float* bg, const BlendFwdOut& out,
                      unsigned long long* counters, cudaStream_t s);

struct BlendBwdIn {
  const float* d_rgb;
  const float* d_depth_acc;
  const float* d_depth_exp;
  const float* d_alpha;
  const float* T_final;
  const uint32_t* n_contrib;
  const float2* D_state;
};
void launch_blend_bwd(const Rec* rec, const uint32_t* pair_vals, const uint2* ranges, const CamBatch& cams,
                      const float* bg, const BlendBwdIn& in, Grad2D* g2d, float* g_aff, int absgrad,
                      unsigned long long* counters, cudaStream_t s);

}  // namespace gsr
