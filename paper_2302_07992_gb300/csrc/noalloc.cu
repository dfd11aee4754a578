// noalloc.cu -- rdhei_extract_noalloc: the K2 receiver's extraction for one image,
// for callers that cannot allocate device memory at all (no cudaMalloc, no caching
// allocator, no workspace handed in): code running inside a host callback or under a
// runtime that owns every allocation, or a tool that links only this library.
//
// Its scratch lives in a file-scope __device__ array that the CUDA runtime sets up when
// the module loads; every GPU that loads the library keeps it until the process exits.
// Host code cannot use the array's name as a device address, so the first call on each
// device looks the address up with cudaGetSymbolAddress (with that device current) and
// caches it; make that first call before any stream capture.  All calls share the one
// array and it keeps the last call's contents: the parts that must start at zero are
// cleared on every call, and calls whose work overlaps on the GPU race on the array.
// The kernels are the ones rdhei_extract launches (hide.cu); a last one-thread kernel
// copies the array's device error word into info->status.  A call on a stream that is
// being captured is refused: the descriptor it uploads lives on the host stack.
#include <atomic>
#include <cstring>

#include "../../include/rdhei.h"
#include "common.cuh"

namespace rdhei {
void launch_count(const Batch& B, bool extract, cudaStream_t st);
void launch_scan(const Batch& B, bool extract, cudaStream_t st);
void launch_z2_xor(const Batch& B, bool decrypt, cudaStream_t st);
}  // namespace rdhei

using namespace rdhei;

namespace {

constexpr uint64_t kMaxPixels = RDHEI_NOALLOC_MAX_PIXELS;
constexpr uint32_t kMaxChunks = (uint32_t)((kMaxPixels + CHUNK_PX - 1) / CHUNK_PX);
// layout of the scratch array
constexpr size_t kZeroBytes = 256;          // error word, tickets, counters: cleared per call
constexpr size_t kDescOff = 256;            // one ImgDesc
constexpr size_t kPrefixOff = 768;          // chunk / K2-block / strip prefix pairs
constexpr size_t kStatusOff = 1024;         // per-chunk slot counts and offsets
constexpr size_t kScratchBytes = kStatusOff + 8 * (size_t)kMaxChunks;
static_assert(sizeof(ImgDesc) <= kPrefixOff - kDescOff, "descriptor does not fit its slot");

__device__ __align__(256) uint8_t g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
// device address of the array per device; host threads may race on the first call of a
// device, and every one of them stores the same address
std::atomic<void*> g_scratch_ptr[kMaxDevices];

// the device error word of the call (index checks of the checked build) into the
// image's info->status
__global__ void k_noalloc_status(const uint32_t* err, rdhei_info* info) { info->status = (int32_t)*err; }

struct Upload {
  ImgDesc d;
  uint8_t pad[kPrefixOff - kDescOff - sizeof(ImgDesc)];
  uint32_t prefix[6];   // chunk_prefix[2], z2_prefix[2], strip_prefix[2]
};

uint32_t le32(const uint8_t* p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

}  // namespace

extern "C" int rdhei_extract_noalloc(const rdhei_job* job, void* stream) {
  if (!job) return RDHEI_EINVAL;
  NvtxRange range("rdhei_extract_noalloc");
  const rdhei_job& j = *job;
  if (j.H < 1 || j.W < 1 || (j.variant < RDHEI_EMR || j.variant > RDHEI_LMR_MED)) return RDHEI_EINVAL;
  const uint64_t N = (uint64_t)j.H * (uint64_t)j.W;
  if (N > kMaxPixels) return RDHEI_ESPACE;                      // beyond the static scratch
  const int bmax = (j.variant & 1) == RDHEI_EMR ? 7 : 8;
  if (j.b != 0 && (j.b < 2 || j.b > bmax)) return RDHEI_EINVAL;
  if (!j.src || !j.info || (reinterpret_cast<uintptr_t>(j.info) & 7)) return RDHEI_EINVAL;
  if (j.max_bits && (!j.bits_out || (reinterpret_cast<uintptr_t>(j.bits_out) & 3))) return RDHEI_EINVAL;
  if ((j.variant & 1) == RDHEI_LMR && (!j.map_bits || (reinterpret_cast<uintptr_t>(j.map_bits) & 3))) return RDHEI_EINVAL;

  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return RDHEI_ECUDA;
  if (cap != cudaStreamCaptureStatusNone) return RDHEI_EINVAL;   // the upload below reads a stack buffer
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RDHEI_ECUDA;
  void* sp = g_scratch_ptr[dev].load(std::memory_order_acquire);
  if (!sp) {
    if (cudaGetSymbolAddress(&sp, g_scratch) != cudaSuccess || !sp) return RDHEI_ECUDA;
    g_scratch_ptr[dev].store(sp, std::memory_order_release);
  }
  uint8_t* base = static_cast<uint8_t*>(sp);

  Upload up;
  std::memset(&up, 0, sizeof(up));
  ImgDesc& d = up.d;
  d.src = j.src;
  d.map_bits = j.map_bits;
  d.bits_out = j.bits_out;
  d.max_bits = j.max_bits < 7 * N ? j.max_bits : 7 * N;
  d.info = j.info;
  d.H = j.H; d.W = j.W; d.variant = j.variant & 1; d.b = j.b;   // extraction is the same for both predictors
  d.one = 1;
  d.nchunks = (uint32_t)((N + CHUNK_PX - 1) / CHUNK_PX);
  for (int k = 0; k < 8; k++) d.k2[k] = le32(j.k2 + 4 * k);
  for (int k = 0; k < 3; k++) d.n2[k] = le32(j.nonce2 + 4 * k);
  const uint32_t z2 = (uint32_t)((d.max_bits + 511) / 512);
  up.prefix[0] = 0; up.prefix[1] = d.nchunks;
  up.prefix[2] = 0; up.prefix[3] = z2;
  up.prefix[4] = 0; up.prefix[5] = 0;

  if (cudaMemsetAsync(base, 0, kZeroBytes, st) != cudaSuccess) return RDHEI_ECUDA;
  if (cudaMemcpyAsync(base + kDescOff, &up, sizeof(up), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return RDHEI_ECUDA;

  Batch B;
  std::memset(&B, 0, sizeof(B));
  B.desc = reinterpret_cast<const ImgDesc*>(base + kDescOff);
  B.chunk_prefix = reinterpret_cast<const uint32_t*>(base + kPrefixOff);
  B.z2_prefix = reinterpret_cast<const uint32_t*>(base + kPrefixOff + 8);
  B.strip_prefix = reinterpret_cast<const uint32_t*>(base + kPrefixOff + 16);
  B.n_images = 1;
  B.total_chunks = d.nchunks;
  B.total_z2_blocks = z2;
  B.err = reinterpret_cast<uint32_t*>(base);
  B.tickets = reinterpret_cast<uint32_t*>(base + 16);
  B.hist_acc = reinterpret_cast<uint32_t*>(base + 64);
  B.chunk_status = reinterpret_cast<unsigned long long*>(base + kStatusOff);
  launch_count(B, true, st);
  launch_scan(B, true, st);
  launch_z2_xor(B, true, st);
  k_noalloc_status<<<1, 1, 0, st>>>(B.err, j.info);
  return cudaGetLastError() == cudaSuccess ? RDHEI_OK : RDHEI_ECUDA;
}
