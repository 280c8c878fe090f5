// gsr_sort_pairs_u32_noalloc: the radix sort of gsr_sort_pairs_u32 for callers that must not
// allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not allowed or not wanted, e.g. a render
// or training step being recorded into a CUDA graph (an allocation cannot be captured and
// cudaMalloc may synchronise the device), a real-time loop that has to keep a fixed memory
// footprint, or a host callback inside another framework's allocator. Such a caller has no
// gsr_ctx workspace to grow, so this entry point takes its scratch (ping-pong buffers, digit
// histograms, look-back status words, block counters) from one array that lives in this
// file as a __device__ global of fixed size. Every GPU that loads the library reserves it
// until the process exits.
#include <algorithm>
#include <mutex>

#include "../../include/gsr.h"
#include "gsr_internal.cuh"

using namespace gsr;

namespace {

// Largest n this entry point accepts: 2^18 pairs.
constexpr long long kMaxN = 1ll << 18;
constexpr long long kMaxTiles = (kMaxN + kSortTile - 1) / kSortTile;
// Layout in 32-bit words; the look-back status words are 64-bit, so their offset is even.
constexpr int kNoAllocBlocks = 64;  // resident blocks per launch: ceil(n / 4096) <= 64 for n <= 2^18
constexpr size_t kKeysTmp = 0;
constexpr size_t kValsTmp = kKeysTmp + kMaxN;
constexpr size_t kHist = kValsTmp + kMaxN;  // digit counts and block counters
constexpr size_t kStatus = (kHist + kSortCountWords + 1) & ~static_cast<size_t>(1);
constexpr size_t kWords = kStatus + 2 * 4 * kMaxTiles * 256;  // 656,388 words, about 2.6 MB
static_assert(kStatus % 2 == 0, "64-bit status words need an even word offset");

static __device__ __align__(256) uint32_t g_sort_scratch[kWords];

std::mutex g_mu;
constexpr int kMaxDevices = 64;
uint32_t* g_scratch_addr[kMaxDevices] = {};

// Device address of g_sort_scratch on the current device, looked up once per device. In host
// code the symbol's name is only a host-side stand-in, so the address must come from
// cudaGetSymbolAddress with that device current. The address is kept for the life of the
// process: after a cudaDeviceReset the module is loaded again and the kept address is stale, so
// a process that resets a device must not call this entry point again on it.
gsr_status scratch_address(uint32_t** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return GSR_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return GSR_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_sort_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return GSR_ERR_CUDA;
    }
    g_scratch_addr[dev] = static_cast<uint32_t*>(p);
  }
  *out = g_scratch_addr[dev];
  return GSR_OK;
}

}  // namespace

extern "C" gsr_status gsr_sort_pairs_u32_noalloc(const uint32_t* keys_in, const uint32_t* vals_in,
                                                 uint32_t* keys_out, uint32_t* vals_out, int64_t n,
                                                 int32_t begin_bit, int32_t end_bit, int32_t* device_err,
                                                 gsr_stream stream) {
  if (n < 0 || begin_bit < 0 || end_bit > 32 || end_bit < begin_bit) return GSR_ERR_INVALID_ARG;
  if (!device_err) return GSR_ERR_INVALID_ARG;  // a timeout must have somewhere to be reported
  if (n > kMaxN) return GSR_ERR_UNSUPPORTED;
  if (n == 0) return GSR_OK;
  if (!keys_in || !vals_in || !keys_out || !vals_out) return GSR_ERR_INVALID_ARG;
  if (keys_out == keys_in || vals_out == vals_in) return GSR_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (end_bit == begin_bit) {
    cudaError_t e = cudaMemcpyAsync(keys_out, keys_in, 4 * n, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(vals_out, vals_in, 4 * n, cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? GSR_OK : GSR_ERR_CUDA;
  }
  uint32_t* base = nullptr;
  const gsr_status st = scratch_address(&base);
  if (st != GSR_OK) return st;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return GSR_ERR_CUDA;
  }
  SortScratch sc;
  sc.keys_tmp = base + kKeysTmp;
  sc.vals_tmp = base + kValsTmp;
  sc.hist = base + kHist;
  sc.status = reinterpret_cast<unsigned long long*>(base + kStatus);
  sc.grid_cap = std::min(2 * sms, kNoAllocBlocks);
  int* err = reinterpret_cast<int*>(device_err);
  // Every call clears the look-back status words, the digit counts and the block counters with
  // stream-ordered memsets before its first kernel (no allocation); the ping-pong buffers need
  // no clearing.
  radix_sort_u32(keys_in, vals_in, keys_out, vals_out, nullptr, n, begin_bit, end_bit, sc, 1u, true, false, err, s);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GSR_OK : GSR_ERR_CUDA;
}
