// common.cuh -- device-side descriptors, keystream and small helpers shared by the
// sm_103a kernels of the multi-MSB replacement RDHEI path (arXiv 2302.07992).
//
// Work decomposition used by every kernel:
//   * images are cut into 64 x 64 tiles (T = 2^6), ragged at the right/bottom edge;
//     the composed block rotation of Eq. (roration) maps aligned 2^k tiles onto
//     aligned 2^k tiles, so tile = unit of gather;
//   * the keystream s (Sec. "Secret key generation") is ChaCha20 (RFC 8439), one
//     64-byte block per 64-pixel tile row when W is a multiple of 64;
//   * raster-order scans (payload offsets of Sec. III-A-2) are reduce-then-scan over
//     8192-pixel chunks (separable calls) or start from per-strip offsets that the
//     top-level pass derives from per-tile label counts (fused calls); no kernel waits
//     for another CTA on this path.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

namespace rdhei {

// Programmatic dependent launch (sm_90+).  The kernels of one operation are launched
// with programmatic stream serialisation: a kernel's CTAs may be scheduled while the
// previous kernel's last CTAs still run.  Every such kernel calls pdl_wait() before it
// reads or writes anything the previous kernel touches (the wait returns once that
// grid has completed and its writes are visible; at once when there is no programmatic
// predecessor), and pdl_trigger() only after its own wait, so that a kernel that
// starts early finds every kernel before its predecessor complete.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Host-side NVTX range for the lifetime of a scope (one ABI call or one stage); with
// no profiler attached a push / pop is a check of an unset function pointer.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

constexpr int TILE = 64;                 // tile side (pixels)
constexpr int TILE_PX = TILE * TILE;
constexpr int SUBTREE_BYTES = 352;       // packed 2-bit angles of levels 1..6 (342 used)
constexpr int AUX_BYTES = 512;           // one bit per tile pixel, tile-major
constexpr int CHUNK_PX = 8192;           // raster chunk of the payload scans
constexpr int ROWVAL_BYTES = 64;         // per-tile row carries of the recovery scan
constexpr int NO_ROTATION = 99;          // lmin value that disables every level

// Offsets of the six levels inside a tile's subtree (row-major per level,
// (64 >> L) x (64 >> L) entries, 2 bits each, entry e at bits 2(e % 4) of byte e / 4).
__host__ __device__ constexpr int subtree_off(int L) {
  return L == 1 ? 0 : L == 2 ? 256 : L == 3 ? 320 : L == 4 ? 336 : L == 5 ? 340 : 341;
}

// Per-image descriptor, built on the host from an rdhei_job plus the workspace layout.
struct ImgDesc {
  const uint8_t* src;
  uint8_t* dst;
  uint8_t* map_bits;
  uint8_t* eta_bits;
  const uint8_t* side_bits;
  uint64_t side_nbits;
  const uint8_t* payload;
  uint64_t nbits;
  uint8_t* bits_out;
  uint64_t max_bits;
  void* info;                 // rdhei_info*
  uint8_t* stash;             // N_px bytes: keystream (encode) / decrypted image (decode)
  uint8_t* ebuf;              // hider: the K2-encrypted message, ceil(nbits / 32) words
  int32_t H, W, variant, b;   // variant: RDHEI_EMR / RDHEI_LMR layout; b: 0 = from info or auto
  int32_t lmin, nlev;         // effective smallest level (NO_ROTATION = none), n
  int32_t med;                // 1: MED predictor (related-work variant) instead of the glide
  uint32_t wave_base, wave_tx;   // MED recovery: first wavefront tile, wavefront tiles per row
  uint32_t one;               // always 1 (a run-time value: see add_fma)
  uint32_t tiles_x, tiles_y, tile_base, chunk_base, nchunks;
  uint32_t k1[8], n1[3], k2[8], n2[3];
};

// Per-tile map entry written by the top-level pass.
struct TileMap {
  uint32_t enc_src;   // encode: for output tile Q, its source tile P
  uint32_t dec_dst;   // decode: for original tile P, its rotated tile Q
  uint8_t enc_shi;    // sum of the angles above level 6 enclosing enc_src (mod 4)
  uint8_t dec_shi;    // the same for P itself
  uint8_t pad[6];
};

// Workspace-wide pointers (device addresses), passed by value to every kernel.
struct Batch {
  const ImgDesc* desc;
  const uint32_t* tile_prefix;    // n + 1 entries: first global tile of each image
  const uint32_t* chunk_prefix;   // n + 1 entries
  const uint32_t* z2_prefix;      // n + 1 entries: first K2 keystream block of each image
  const uint32_t* strip_prefix;   // n + 1 entries: first 64-row strip of each image
  const uint32_t* tile_owner;     // total_tiles entries: image of each global tile
  const uint32_t* strip_owner;    // total_strips entries: image of each global strip
  uint32_t total_strips;
  uint32_t total_z2_blocks;
  int n_images;
  uint32_t total_tiles, total_chunks;
  uint32_t* err;                  // workspace error word
  uint32_t* tickets;              // 8 dispenser counters (zeroed per call)
  uint32_t* hist_acc;             // n * 16 counters (zeroed per call)
  unsigned long long* chunk_status;   // total_chunks (zeroed per call)
  uint32_t* tile_flags;           // total_tiles (zeroed per call)
  uint8_t* tile_rows;             // total_tiles * 128: aggregate + inclusive row carries
  uint8_t* subtree;               // total_tiles * SUBTREE_BYTES
  uint8_t* aux;                   // total_tiles * AUX_BYTES
  uint8_t* sigma6;                // total_tiles
  TileMap* tilemap;               // total_tiles
  uint8_t* lab;                   // MED decode: total_tiles * AUX_BYTES de-rotated label bits
  uint32_t* wave_flags;           // MED decode: total_wave done flags (zeroed per call)
  const uint2* wave_list;         // MED decode: (image, ty << 16 | tx) in anti-diagonal order
  uint32_t total_wave;
  int32_t wave_cols;              // MED decode: 0 = row-band pipeline, else tile width (64, 128, 256)
  uint16_t* tile_cnt;             // total_tiles * 8: label-0 pixels per tile (owner: b = 1..8; receiver: [0])
  uint32_t* strip_base;           // total_strips: first payload bit of each 64-row strip (fused calls)
  uint32_t* strip_tot;            // total_strips: payload bits of each strip (fused calls)
  uint8_t* rowcnt;                // total_tiles * 64: label-0 pixels of each tile row (split strips)
  uint32_t* part_base;            // total_strips * 16: first payload bit of each part of a strip
  int32_t part_rows;              // fused decode: rows of a strip per extraction CTA (64, 32, .., 4)
  int32_t count_rows;             // fused decode: the first pass writes rowcnt
};

constexpr int MAX_PARTS = 16;     // parts of a 64-row strip at 4 rows each

// MED recovery wavefront tile: 32 rows (one warp lane per row) x wave_cols columns.
constexpr int WAVE_ROWS = 32, WAVE_COLS_DEFAULT = 128;

// Median edge detector on four bytes at once (related-work predictor, LOCO-I):
// min(A, B) where C >= max(A, B), max(A, B) where C <= min(A, B), else A + B - C.
// The same value is min + max - clamp(C, min, max), which never leaves [min, max];
// it is computed on the even and the odd bytes as 16-bit lanes with the hardware
// two-lane min / max.
__device__ __forceinline__ uint32_t min_u16x2(uint32_t a, uint32_t b) {
  uint32_t r;
  asm("min.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
__device__ __forceinline__ uint32_t max_u16x2(uint32_t a, uint32_t b) {
  uint32_t r;
  asm("max.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
__device__ __forceinline__ uint32_t med2(uint32_t a, uint32_t b, uint32_t c) {   // two 16-bit lanes
  const uint32_t mn = min_u16x2(a, b), mx = max_u16x2(a, b);
  return mn + mx - min_u16x2(max_u16x2(c, mn), mx);                              // no lane carries
}
__device__ __forceinline__ uint32_t med4(uint32_t A, uint32_t Bv, uint32_t C) {
  const uint32_t M = 0x00FF00FFu;
  return med2(A & M, Bv & M, C & M) | (med2((A >> 8) & M, (Bv >> 8) & M, (C >> 8) & M) << 8);
}

// Error codes shared with rdhei.h.
constexpr int ERR_CAPACITY = 2;
constexpr int ERR_TIMEOUT = 4;
constexpr int ERR_BOUNDS = 6;

// ------------------------------------------------------------------------------------
// ChaCha20 block function (RFC 8439 Sec. 2.3), 20 rounds, written for the GPU: the 16
// state words stay in registers; rotations are funnel shifts.  The XORs and rotations
// occupy the integer/logic pipe, so the additions go to the FMA pipe as integer
// multiply-adds a * one + b, with `one` a run-time 1 (ImgDesc::one) that the compiler
// cannot fold back into a plain add.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t rotl32(uint32_t x, int n) { return __funnelshift_l(x, x, n); }
__device__ __forceinline__ uint32_t add_fma(uint32_t a, uint32_t b, uint32_t one) { return a * one + b; }

#define RDHEI_QR(a, b, c, d)                               \
  a = add_fma(a, b, one); d ^= a; d = rotl32(d, 16);       \
  c = add_fma(c, d, one); b ^= c; b = rotl32(b, 12);       \
  a = add_fma(a, b, one); d ^= a; d = rotl32(d, 8);        \
  c = add_fma(c, d, one); b ^= c; b = rotl32(b, 7);

// UNROLL: double rounds unrolled per loop iteration (10 = straight-line code; kernels
// with much other code keep their instruction footprint small with 2).
template <int UNROLL = 10>
__device__ __forceinline__ void chacha20_block(const uint32_t key[8], uint32_t counter,
                                               const uint32_t nonce[3], uint32_t o[16], uint32_t one) {
  const uint32_t c0 = 0x61707865u, c1 = 0x3320646eu, c2 = 0x79622d32u, c3 = 0x6b206574u;
  uint32_t x0 = c0, x1 = c1, x2 = c2, x3 = c3;
  uint32_t x4 = key[0], x5 = key[1], x6 = key[2], x7 = key[3];
  uint32_t x8 = key[4], x9 = key[5], x10 = key[6], x11 = key[7];
  uint32_t x12 = counter, x13 = nonce[0], x14 = nonce[1], x15 = nonce[2];
#pragma unroll UNROLL
  for (int i = 0; i < 10; i++) {
    RDHEI_QR(x0, x4, x8, x12) RDHEI_QR(x1, x5, x9, x13) RDHEI_QR(x2, x6, x10, x14) RDHEI_QR(x3, x7, x11, x15)
    RDHEI_QR(x0, x5, x10, x15) RDHEI_QR(x1, x6, x11, x12) RDHEI_QR(x2, x7, x8, x13) RDHEI_QR(x3, x4, x9, x14)
  }
  o[0] = add_fma(x0, c0, one); o[1] = add_fma(x1, c1, one); o[2] = add_fma(x2, c2, one);
  o[3] = add_fma(x3, c3, one);
  o[4] = add_fma(x4, key[0], one); o[5] = add_fma(x5, key[1], one); o[6] = add_fma(x6, key[2], one);
  o[7] = add_fma(x7, key[3], one); o[8] = add_fma(x8, key[4], one); o[9] = add_fma(x9, key[5], one);
  o[10] = add_fma(x10, key[6], one); o[11] = add_fma(x11, key[7], one);
  o[12] = add_fma(x12, counter, one); o[13] = add_fma(x13, nonce[0], one);
  o[14] = add_fma(x14, nonce[1], one); o[15] = add_fma(x15, nonce[2], one);
}
#undef RDHEI_QR

// ------------------------------------------------------------------------------------
// small helpers
// ------------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;  // 2 s bound on any device-side wait

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Asynchronous global -> shared copies (cp.async): commit and wait for the groups.
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void set_error(uint32_t* err, int code) { atomicCAS(err, 0u, (uint32_t)code); }

// Index checks of the checked build (-DRDHEI_CHECK, a stand-in for a memory checker):
// a failing check records ERR_BOUNDS in the workspace error word and the caller skips
// the access.  The normal build compiles every check to `true`.
#ifdef RDHEI_CHECK
__device__ __forceinline__ bool idx_ok(uint32_t* err, bool cond) {
  if (!cond) set_error(err, ERR_BOUNDS);
  return cond;
}
#define RDHEI_IDX_OK(err, cond) ::rdhei::idx_ok((err), (cond))
#else
#define RDHEI_IDX_OK(err, cond) true
#endif

// Image index owning global tile / chunk `g` (binary search in a prefix array).
__device__ __forceinline__ int owner_of(const uint32_t* prefix, int n, uint32_t g) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (__ldg(prefix + mid) <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__host__ __device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }

__device__ __forceinline__ uint32_t bswap32(uint32_t x) { return __byte_perm(x, 0, 0x0123); }

// Quarter-turn of one coordinate bit pair (u = row bit, v = column bit) by `a`
// counter-clockwise turns: one turn maps (u, v) -> (1 - v, u).  Encoded as a 32-bit
// table: entry (a, u, v) at bits 2 * (4a + 2u + v), value (u' << 1) | v'.
//   a=0: 00->00 01->01 10->10 11->11
//   a=1: 00->10 01->00 10->11 11->01
//   a=2: 00->11 01->10 10->01 11->00
//   a=3: 00->01 01->11 10->00 11->10
constexpr uint32_t ROT_FWD_LUT =
    (0u << 0) | (1u << 2) | (2u << 4) | (3u << 6) |
    (2u << 8) | (0u << 10) | (3u << 12) | (1u << 14) |
    (3u << 16) | (2u << 18) | (1u << 20) | (0u << 22) |
    (1u << 24) | (3u << 26) | (0u << 28) | (2u << 30);
// inverse turn: (a, u', v') -> (u, v)
constexpr uint32_t ROT_INV_LUT =
    (0u << 0) | (1u << 2) | (2u << 4) | (3u << 6) |
    (1u << 8) | (3u << 10) | (0u << 12) | (2u << 14) |
    (3u << 16) | (2u << 18) | (1u << 20) | (0u << 22) |
    (2u << 24) | (0u << 26) | (3u << 28) | (1u << 30);

__host__ __device__ __forceinline__ uint32_t rot_bits(uint32_t lut, uint32_t a, uint32_t uv) {
  return (lut >> (2u * (((a & 3u) << 2) | uv))) & 3u;
}

// Up to 32 bits of an MSB-first stream starting at bit `pos`, returned LSB-first
// (bit c = stream bit pos + c); `nwords` bounds the 32-bit words that may be read.
// 32-bit positions: an image holds at most 2^27 pixels, its streams at most 2^30 bits.
__device__ __forceinline__ uint32_t stream_bits32(const uint8_t* s, uint32_t nwords, uint32_t pos) {
  const uint32_t* w = reinterpret_cast<const uint32_t*>(s);
  const uint32_t wi = pos >> 5;
  uint32_t sh = (uint32_t)(pos & 31);
  uint32_t w0 = wi < nwords ? bswap32(__ldg(w + wi)) : 0u;
  uint32_t w1 = (sh && wi + 1 < nwords) ? bswap32(__ldg(w + wi + 1)) : 0u;
  uint32_t msb = sh ? (w0 << sh) | (w1 >> (32 - sh)) : w0;
  return __brev(msb);
}

// The same from a stream that the calling kernel itself wrote earlier (coherent
// L2 loads: the read-only path may not be used for data written by the same kernel).
__device__ __forceinline__ uint32_t stream_bits32_cg(const uint8_t* s, uint32_t nwords, uint32_t pos) {
  const uint32_t* w = reinterpret_cast<const uint32_t*>(s);
  const uint32_t wi = pos >> 5;
  uint32_t sh = (uint32_t)(pos & 31);
  uint32_t w0 = wi < nwords ? bswap32(__ldcg(w + wi)) : 0u;
  uint32_t w1 = (sh && wi + 1 < nwords) ? bswap32(__ldcg(w + wi + 1)) : 0u;
  uint32_t msb = sh ? (w0 << sh) | (w1 >> (32 - sh)) : w0;
  return __brev(msb);
}

}  // namespace rdhei
