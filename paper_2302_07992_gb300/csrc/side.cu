// side.cu -- LMR side information (Sec. III-B-1, "Maps generation, rotation, and
// compression", "Maps embedding"): lossless bi-level compression of the rotated
// first-MSB map rot(eta) and the rotated location map rot(l), the container that
// carries both in the first MSB plane, and a device kernel that packs that plane.
//
// The paper uses JBIG-KIT.  This coder is JBIG-style, of this project's design:
//   context   10 causal neighbours: row y-2 at x-1, x, x+1; row y-1 at x-2 .. x+2;
//             row y at x-2, x-1 (listed from the most significant context bit down);
//             outside the bitmap reads 0;
//   model     per context, counts c0, c1 start at 1 and grow by 2 per coded symbol
//             (Krichevsky-Trofimov); when c0 + c1 > 8192 both become (c >> 1) | 1;
//   coder     binary arithmetic coding after Witten, Neal and Cleary (1987): 32-bit
//             low/high, symbol 0 takes the lower floor(range * c0 / (c0 + c1)) values,
//             pending ("follow") bits for the middle-half case, two terminating bits,
//             MSB-first bytes padded with zeros.
// Container: byte 0 = b; bytes 1..4 and 5..8 = byte lengths of the rot(eta) and rot(l)
// streams (big-endian); then the two streams.  It must fit into H * W bits.
//
// Host code runs the coder per image on a pool of std::threads; the context of each
// pixel is updated incrementally from three sliding row windows.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <thread>
#include <vector>

#include "../../include/rdhei.h"
#include "common.cuh"

namespace {

constexpr uint32_t HALF = 1u << 31, QUARTER = 1u << 30;
constexpr uint32_t COUNT_LIMIT = 8192;
constexpr int HEADER = 9;

inline int get_bit(const uint8_t* p, uint64_t k) { return (p[k >> 3] >> (7 - (k & 7))) & 1; }

struct Model {
  uint16_t c0[1024], c1[1024];
  Model() {
    for (int i = 0; i < 1024; i++) c0[i] = c1[i] = 1;
  }
  inline void update(int ctx, int bit) {
    if (bit) c1[ctx] += 2; else c0[ctx] += 2;
    if ((uint32_t)c0[ctx] + c1[ctx] > COUNT_LIMIT) {
      c0[ctx] = (uint16_t)((c0[ctx] >> 1) | 1);
      c1[ctx] = (uint16_t)((c1[ctx] >> 1) | 1);
    }
  }
};

// Row windows: rows unpacked into byte arrays, pixel x at index x + 2, with zeros for
// x < 0 and x >= W (the windows slide one column past the last pixel, reading x + 3).
struct Rows {
  int W;
  std::vector<uint8_t> r0, r1, r2;   // rows y, y-1, y-2
  explicit Rows(int W_) : W(W_), r0(W_ + 6, 0), r1(W_ + 6, 0), r2(W_ + 6, 0) {}
  void advance() {
    std::swap(r2, r1);
    std::swap(r1, r0);
    std::fill(r0.begin(), r0.end(), 0);
  }
};

struct BitWriter {
  uint8_t* out;
  size_t cap_bits, nbits = 0;
  bool overflow = false;
  uint32_t pending = 0;
  BitWriter(uint8_t* o, size_t cap_bytes) : out(o), cap_bits(cap_bytes * 8) {}
  inline void put(int bit) {
    if (nbits >= cap_bits) { overflow = true; return; }
    if ((nbits & 7) == 0) out[nbits >> 3] = 0;
    if (bit) out[nbits >> 3] |= (uint8_t)(0x80u >> (nbits & 7));
    nbits++;
  }
  inline void emit(int bit) {
    put(bit);
    for (; pending; pending--) put(!bit);
  }
};

// Encode an H x W bitmap given as MSB-first packed bits.  Returns the byte length, or
// 0 with *overflow set when the code would not fit into cap bytes.
size_t encode_bitmap(const uint8_t* bits, int H, int W, uint8_t* out, size_t cap, bool* overflow) {
  Model m;
  Rows R(W);
  BitWriter bw(out, cap);
  uint32_t low = 0, high = 0xFFFFFFFFu;
  for (int y = 0; y < H; y++) {
    R.advance();
    const uint64_t row0 = (uint64_t)y * W;
    // r0 of row y is filled as we go; r1, r2 were filled on earlier rows
    int w2 = (R.r2[1] << 2) | (R.r2[2] << 1) | R.r2[3];
    int w1 = (R.r1[0] << 4) | (R.r1[1] << 3) | (R.r1[2] << 2) | (R.r1[3] << 1) | R.r1[4];
    int w0 = 0;
    for (int x = 0; x < W; x++) {
      const int ctx = (w2 << 7) | (w1 << 2) | w0;
      const int bit = get_bit(bits, row0 + x);
      const uint32_t c0 = m.c0[ctx], c1 = m.c1[ctx];
      const uint64_t range = (uint64_t)(high - low) + 1;
      const uint32_t split = low + (uint32_t)(range * c0 / (c0 + c1)) - 1;
      if (bit) low = split + 1; else high = split;
      for (;;) {
        if (high < HALF) {
          bw.emit(0);
        } else if (low >= HALF) {
          bw.emit(1);
          low -= HALF;
          high -= HALF;
        } else if (low >= QUARTER && high < HALF + QUARTER) {
          bw.pending++;
          low -= QUARTER;
          high -= QUARTER;
        } else {
          break;
        }
        low <<= 1;
        high = (high << 1) | 1;
      }
      if (bw.overflow) { *overflow = true; return 0; }
      m.update(ctx, bit);
      R.r0[x + 2] = (uint8_t)bit;
      // slide the windows to x + 1
      w2 = ((w2 << 1) | R.r2[x + 4]) & 7;        // row y-2, x+2 enters (window x..x+2)
      w1 = ((w1 << 1) | R.r1[x + 5]) & 31;       // row y-1, x+3 enters
      w0 = ((w0 << 1) | bit) & 3;                // row y, x enters
    }
  }
  bw.pending++;
  bw.emit(low < QUARTER ? 0 : 1);
  if (bw.overflow) { *overflow = true; return 0; }
  *overflow = false;
  return (bw.nbits + 7) / 8;
}

struct BitReader {
  const uint8_t* in;
  uint64_t nbits, pos = 0;
  BitReader(const uint8_t* p, size_t len) : in(p), nbits((uint64_t)len * 8) {}
  inline uint32_t get() {
    const uint32_t v = pos < nbits ? (uint32_t)get_bit(in, pos) : 0u;
    pos++;
    return v;
  }
};

void decode_bitmap(const uint8_t* in, size_t len, int H, int W, uint8_t* bits) {
  Model m;
  Rows R(W);
  BitReader br(in, len);
  uint32_t low = 0, high = 0xFFFFFFFFu, value = 0;
  for (int i = 0; i < 32; i++) value = (value << 1) | br.get();
  std::memset(bits, 0, ((uint64_t)H * W + 7) / 8);
  for (int y = 0; y < H; y++) {
    R.advance();
    const uint64_t row0 = (uint64_t)y * W;
    int w2 = (R.r2[1] << 2) | (R.r2[2] << 1) | R.r2[3];
    int w1 = (R.r1[0] << 4) | (R.r1[1] << 3) | (R.r1[2] << 2) | (R.r1[3] << 1) | R.r1[4];
    int w0 = 0;
    for (int x = 0; x < W; x++) {
      const int ctx = (w2 << 7) | (w1 << 2) | w0;
      const uint32_t c0 = m.c0[ctx], c1 = m.c1[ctx];
      const uint64_t range = (uint64_t)(high - low) + 1;
      const uint32_t split = low + (uint32_t)(range * c0 / (c0 + c1)) - 1;
      int bit;
      if (value <= split) { bit = 0; high = split; } else { bit = 1; low = split + 1; }
      for (;;) {
        if (high < HALF) {
        } else if (low >= HALF) {
          low -= HALF; high -= HALF; value -= HALF;
        } else if (low >= QUARTER && high < HALF + QUARTER) {
          low -= QUARTER; high -= QUARTER; value -= QUARTER;
        } else {
          break;
        }
        low <<= 1;
        high = (high << 1) | 1;
        value = (value << 1) | br.get();
      }
      m.update(ctx, bit);
      if (bit) bits[(row0 + x) >> 3] |= (uint8_t)(0x80u >> ((row0 + x) & 7));
      R.r0[x + 2] = (uint8_t)bit;
      w2 = ((w2 << 1) | R.r2[x + 4]) & 7;
      w1 = ((w1 << 1) | R.r1[x + 5]) & 31;
      w0 = ((w0 << 1) | bit) & 3;
    }
  }
}

bool valid_size(int H, int W) { return H >= 1 && W >= 1 && (uint64_t)H * W <= (1ull << 27); }

void put_u32(uint8_t* p, uint32_t v) { p[0] = v >> 24; p[1] = v >> 16; p[2] = v >> 8; p[3] = v; }
uint32_t get_u32(const uint8_t* p) { return ((uint32_t)p[0] << 24) | ((uint32_t)p[1] << 16) | ((uint32_t)p[2] << 8) | p[3]; }

int pack_one(rdhei_side_pack_job& j) {
  if (!valid_size(j.H, j.W) || !j.eta_bits || !j.map_bits || !j.side || j.b < 2 || j.b > 8) return RDHEI_EINVAL;
  const size_t cap = ((uint64_t)j.H * j.W) / 8;    // whole bytes of the first MSB plane
  j.side_nbits = 0;
  if (cap < HEADER) return RDHEI_ECAPACITY;
  bool ovf = false;
  const size_t le = encode_bitmap(j.eta_bits, j.H, j.W, j.side + HEADER, cap - HEADER, &ovf);
  if (ovf) return RDHEI_ECAPACITY;
  const size_t ll = encode_bitmap(j.map_bits, j.H, j.W, j.side + HEADER + le, cap - HEADER - le, &ovf);
  if (ovf) return RDHEI_ECAPACITY;
  j.side[0] = (uint8_t)j.b;
  put_u32(j.side + 1, (uint32_t)le);
  put_u32(j.side + 5, (uint32_t)ll);
  j.side_nbits = 8ull * (HEADER + le + ll);
  return RDHEI_OK;
}

int unpack_one(rdhei_side_unpack_job& j) {
  if (!valid_size(j.H, j.W) || !j.plane || !j.eta_bits || !j.map_bits) return RDHEI_EINVAL;
  const uint64_t cap = ((uint64_t)j.H * j.W) / 8;
  if (cap < HEADER) return RDHEI_EINVAL;
  const int b = j.plane[0];
  const uint64_t le = get_u32(j.plane + 1), ll = get_u32(j.plane + 5);
  if (b < 2 || b > 8 || HEADER + le + ll > cap) return RDHEI_EINVAL;
  j.b = b;
  decode_bitmap(j.plane + HEADER, le, j.H, j.W, j.eta_bits);
  decode_bitmap(j.plane + HEADER + le, ll, j.H, j.W, j.map_bits);
  return RDHEI_OK;
}

template <class Job, class Fn>
int run_pool(Job* jobs, int n, int threads, Fn fn) {
  if (n < 0 || (n > 0 && !jobs)) return RDHEI_EINVAL;
  if (threads <= 0) threads = (int)std::max(1u, std::thread::hardware_concurrency());
  threads = std::min(threads, std::max(n, 1));
  std::atomic<int> next{0};
  auto worker = [&]() {
    for (int i = next++; i < n; i = next++) jobs[i].status = fn(jobs[i]);
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < threads; t++) pool.emplace_back(worker);
  worker();
  for (auto& th : pool) th.join();
  return RDHEI_OK;
}

}  // namespace

// ------------------------------------------------------------------ device --
namespace rdhei {
// bit 7 of every pixel, packed MSB-first: one warp turns 32 pixels into one word
__global__ void k_msb_plane(const uint8_t* __restrict__ src, uint64_t npx, uint32_t* __restrict__ out) {
  const uint64_t nwords = (npx + 31) / 32;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nwords * 32; i += stride) {
    const int v = i < npx ? (__ldg(src + i) >> 7) : 0;
    const uint32_t word = __brev(__ballot_sync(0xffffffffu, v));
    if ((threadIdx.x & 31) == 0) out[i >> 5] = bswap32(word);
  }
}
}  // namespace rdhei

extern "C" int rdhei_bilevel_encode(const uint8_t* bits, int H, int W, uint8_t* out, size_t cap, size_t* len) {
  if (!valid_size(H, W) || !bits || !out || !len) return RDHEI_EINVAL;
  bool ovf = false;
  *len = encode_bitmap(bits, H, W, out, cap, &ovf);
  return ovf ? RDHEI_ESPACE : RDHEI_OK;
}

extern "C" int rdhei_bilevel_decode(const uint8_t* in, size_t len, int H, int W, uint8_t* bits) {
  if (!valid_size(H, W) || (!in && len) || !bits) return RDHEI_EINVAL;
  decode_bitmap(in, len, H, W, bits);
  return RDHEI_OK;
}

extern "C" int rdhei_lmr_side_pack(rdhei_side_pack_job* jobs, int n, int threads) {
  rdhei::NvtxRange range("rdhei_lmr_side_pack");
  return run_pool(jobs, n, threads, pack_one);
}

extern "C" int rdhei_lmr_side_unpack(rdhei_side_unpack_job* jobs, int n, int threads) {
  rdhei::NvtxRange range("rdhei_lmr_side_unpack");
  return run_pool(jobs, n, threads, unpack_one);
}

extern "C" int rdhei_msb_plane(const uint8_t* src, int H, int W, uint8_t* out_bits, void* stream) {
  if (!valid_size(H, W) || !src || !out_bits || (reinterpret_cast<uintptr_t>(out_bits) & 3)) return RDHEI_EINVAL;
  const uint64_t npx = (uint64_t)H * W;
  const uint64_t threads = ((npx + 31) / 32) * 32;
  const int block = 256;
  const int grid = (int)std::min<uint64_t>((threads + block - 1) / block, 152ull * 16);
  rdhei::k_msb_plane<<<grid, block, 0, reinterpret_cast<cudaStream_t>(stream)>>>(src, npx,
                                                                                 reinterpret_cast<uint32_t*>(out_bits));
  return cudaGetLastError() == cudaSuccess ? RDHEI_OK : RDHEI_ECUDA;
}

extern "C" size_t rdhei_side_pack_job_size(void) { return sizeof(rdhei_side_pack_job); }
extern "C" size_t rdhei_side_unpack_job_size(void) { return sizeof(rdhei_side_unpack_job); }

// Eq. optimal_b as an ordered candidate list (the owner's fit loop walks it when the
// compressed maps of its first choice do not fit): capacity b * zeros(b) (EMR) or
// (b - 1) * zeros(b) (LMR), zeros(b) = sum over t >= b of hist[t]; decreasing capacity,
// ties to the smaller b.  Insertion sort of at most seven entries.
extern "C" int rdhei_b_candidates(const uint32_t hist[9], int variant, int32_t order[7], uint64_t capacity[7]) {
  if (!hist || !order || !capacity || variant < RDHEI_EMR || variant > RDHEI_LMR_MED) return -1;
  const bool lmr = (variant & 1) == RDHEI_LMR;
  const int bmax = lmr ? 8 : 7;
  int n = 0;
  for (int b = 2; b <= bmax; b++) {
    uint64_t zeros = 0;
    for (int t = b; t <= 8; t++) zeros += hist[t];
    const uint64_t cap = (uint64_t)(lmr ? b - 1 : b) * zeros;
    int k = n++;
    while (k > 0 && capacity[k - 1] < cap) {          // earlier (smaller) b wins ties: strict <
      capacity[k] = capacity[k - 1];
      order[k] = order[k - 1];
      k--;
    }
    capacity[k] = cap;
    order[k] = b;
  }
  return n;
}
