// Allocation-free blind phase search + demap.
//
// Some callers of this library cannot allocate device memory at the point
// where they need carrier recovery: real-time loops that must never hit the
// allocator's implicit device synchronisation (a cudaMalloc can wait for work
// already queued on the device, which breaks their timing), and plugin hosts
// that hand out fixed device memory budgets up front and own every
// allocation.  rx_bps_demap_noalloc serves them: it runs
// the same BPS / unwrap / hard-decision kernels as rx_process on an
// equalised block the caller provides, with all of its scratch in one
// file-scope device array, and never calls cudaMalloc or cudaFree.
//
// The array holds the per-symbol angle bytes and the per-chunk tables for up
// to kNoAllocMaxSymbols symbols per polarisation (about 2.1 MiB); every GPU
// that loads the library keeps it until the process exits.  All calls share
// it, so calls whose work overlaps on the GPU race; run them on one stream or
// order them.  The first call on a device looks up the array's device address
// (cudaGetSymbolAddress, with that device current) and caches it together with
// the device's current context; make that first call before any stream
// capture.  A call that finds a different context (the device was reset and its
// primary context re-created) looks the address up again.
#include <cudaTypedefs.h>
#include <string.h>

#include <mutex>

#include "common.cuh"
#include "rx_internal.h"

namespace rx {
namespace {

constexpr int64_t kNoAllocMaxSymbols = 1 << 20;  // per polarisation
constexpr int kNoAllocChunk = 256;
constexpr int64_t kNoAllocChunks = kNoAllocMaxSymbols / kNoAllocChunk;
// byte layout of the scratch array
constexpr size_t kOffBhat = 0;                                              // int8 [2][max]
constexpr size_t kOffChunkM = kOffBhat + 2 * kNoAllocMaxSymbols;            // int64 [2][chunks]
constexpr size_t kOffChunkR = kOffChunkM + 2 * kNoAllocChunks * 8;          // int32 [2][chunks]
constexpr size_t kOffChunkS2 = kOffChunkR + 2 * kNoAllocChunks * 4;         // float [2][chunks]
constexpr size_t kOffCarry = kOffChunkS2 + 2 * kNoAllocChunks * 4;          // int64 [2]
constexpr size_t kOffRegion = kOffCarry + 256;                              // double [2]
constexpr size_t kScratchBytes = kOffRegion + 256;

constexpr int kMaxDevices = 64;
struct ScratchRef {
  void *ctx;            // the context the address belongs to
  unsigned char *addr;  // device address of the array, from the symbol lookup
};
ScratchRef g_scratch[kMaxDevices] = {};
std::mutex g_scratch_mu;

// The calling thread's current context (driver entry point fetched through the
// runtime, so the library needs no link against the driver library); nullptr
// if it cannot be had.
void *current_context() {
  static PFN_cuCtxGetCurrent_v4000 fn = nullptr;
  static bool looked = false;
  if (!looked) {
    looked = true;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
  }
  CUcontext c = nullptr;
  if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
  return c;
}

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

}  // namespace rx

using namespace rx;

extern "C" rx_status rx_bps_demap_noalloc(const float *y, int64_t y_stride, int64_t n_symbols, int bits_per_symbol,
                                          int bps_halfwin, uint32_t *bits, int64_t bits_stride, void *cuda_stream) {
  if (!y || !bits || n_symbols < 0 || y_stride < n_symbols || bits_stride * 32 < n_symbols * bits_per_symbol)
    return RX_EINVAL;
  if (n_symbols > kNoAllocMaxSymbols) return RX_EINVAL;  // beyond the scratch array
  if (bits_per_symbol != 2 && bits_per_symbol != 4) return RX_EUNSUPPORTED;
  if (bps_halfwin < 0 || bps_halfwin > 64) return RX_EUNSUPPORTED;
  if ((uintptr_t)y % 8) return RX_EINVAL;
  if (n_symbols == 0) return RX_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RX_ECUDA;
  unsigned char *base;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    ScratchRef &ref = g_scratch[dev];
    if (!ref.addr || (ref.ctx != nullptr && current_context() != ref.ctx)) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return RX_ECUDA;
      ref.addr = static_cast<unsigned char *>(p);
      ref.ctx = current_context();   // the lookup made the device's context current
    }
    base = ref.addr;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  // the unwrap count starts at zero for every call
  if (cudaMemsetAsync(base + kOffCarry, 0, 2 * sizeof(int64_t), s) != cudaSuccess) return RX_ECUDA;
  BpsLaunch B;
  memset(&B, 0, sizeof(B));
  B.y = reinterpret_cast<const float2 *>(y);
  B.y_base = 0;
  B.y_stride = y_stride;
  B.bhat = reinterpret_cast<int8_t *>(base + kOffBhat);
  B.bh_base = 0;
  B.bh_stride = kNoAllocMaxSymbols;
  B.chunk = kNoAllocChunk;
  B.n_chunks = (n_symbols + kNoAllocChunk - 1) / kNoAllocChunk;
  B.chunk_m = reinterpret_cast<int64_t *>(base + kOffChunkM);
  B.chunk_r = reinterpret_cast<int *>(base + kOffChunkR);
  B.chunk_s2 = reinterpret_cast<float *>(base + kOffChunkS2);
  B.m_carry = reinterpret_cast<int64_t *>(base + kOffCarry);
  B.region_s2 = reinterpret_cast<double *>(base + kOffRegion);
  B.k_lo = 0;
  B.k_hi = n_symbols;
  B.K_end = n_symbols;  // the block is the whole stream: windows truncate at both ends
  B.A = n_symbols;      // one region
  B.span = n_symbols;
  B.Nb = bps_halfwin;
  B.mod_bits = bits_per_symbol;
  B.need_s2 = 0;        // hard bits only
  B.bits = bits;
  B.bits_stride = bits_stride;
  B.out_first = 0;
  return launch_bps(B, s) == cudaSuccess ? RX_OK : RX_ECUDA;
}
