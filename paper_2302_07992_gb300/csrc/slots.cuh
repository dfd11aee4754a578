// slots.cuh -- the payload slots of Sec. III-A-2 / III-B-2 (hider) and Sec. III-A-3 /
// III-B-3 (K2 receiver): label-0 pixels, visited in raster order of the rotated image,
// each hold b (EMR) or b - 1 (LMR) bits of the K2-encrypted message back to back,
// first bit in bit 7 (EMR) or bit 6 (LMR).  Shared by the separable scan kernels
// (hide.cu) and the fused owner-and-hider kernel (encode.cu).
//
// A thread owns 32 consecutive pixels of a raster chunk of 8192; a block scan of the
// per-thread slot counts gives each thread's first slot inside the chunk.
//   spread_slots:  message stream -> slot fields of my pixels (hider);
//   gather_slots:  slot fields of my pixels -> chunk-local stream (receiver).
// Per 4-pixel word the fields move with one byte permute (the label-0 pattern of the
// word selects it) and integer multiply-adds that place each field (k + 1)(8 - s) bits
// further up -- no per-pixel loop.
#pragma once
#include "common.cuh"
#include "../../include/rdhei.h"

namespace rdhei {

constexpr int HIDE_THREADS = 256;
constexpr int HIDE_PX = 32;                          // pixels per thread
constexpr int SCAN_PX = HIDE_THREADS * HIDE_PX;      // 8192 pixels per chunk
static_assert(SCAN_PX == CHUNK_PX, "chunk size shared with the host layout");
constexpr int SBUF_WORDS = 7 * SCAN_PX / 32 + 4;     // slots of one chunk, in 32-bit words

// n (1..32) bits of an MSB-first word array starting at bit idx, right-aligned
__device__ __forceinline__ uint32_t get_bits(const uint32_t* buf, uint32_t idx, uint32_t n) {
  const uint32_t w = idx >> 5, sh = idx & 31;
  const uint64_t v = ((uint64_t)buf[w] << 32) | buf[w + 1];
  return (uint32_t)((v << sh) >> (64 - n));
}
// OR n (1..32) right-aligned bits into an MSB-first shared word array at bit idx
__device__ __forceinline__ void or_bits(uint32_t* buf, uint32_t idx, uint32_t val, uint32_t n) {
  const uint32_t w = idx >> 5, sh = idx & 31;
  const uint64_t run = (((uint64_t)val) << (64 - n)) >> sh;
  const uint32_t hi = (uint32_t)(run >> 32), lo = (uint32_t)run;
  if (hi) atomicOr(buf + w, hi);
  if (lo) atomicOr(buf + w + 1, lo);
}

// My 32 pixels of a chunk (raw words, loads in flight until first use) and the mask
// of the redundant (label-0) ones: EMR reads the map from the LSB plane, LMR from the
// packed rotated map.
struct ChunkPx {
  uint32_t px[8];
  uint32_t lbits;   // LMR: packed map bits of my 32 pixels
  int valid;
};

__device__ __forceinline__ void issue_chunk(const ImgDesc& d, uint32_t c, int t, bool need_px, ChunkPx& r) {
  const uint64_t N = (uint64_t)d.H * d.W;
  const uint64_t p0 = (uint64_t)c * SCAN_PX + (uint64_t)HIDE_PX * t;
  r.valid = p0 < N ? (int)umin64(HIDE_PX, N - p0) : 0;
#pragma unroll
  for (int i = 0; i < 8; i++) r.px[i] = 0;
  r.lbits = 0xFFFFFFFFu;
  const bool lmr = d.variant == RDHEI_LMR;
  if (need_px || !lmr) {
    const uint8_t* src = d.src + p0;
    if (r.valid == HIDE_PX && ((reinterpret_cast<uintptr_t>(src) & 15) == 0)) {
      const uint4 a = __ldcs(reinterpret_cast<const uint4*>(src)), e = __ldcs(reinterpret_cast<const uint4*>(src + 16));
      r.px[0] = a.x; r.px[1] = a.y; r.px[2] = a.z; r.px[3] = a.w;
      r.px[4] = e.x; r.px[5] = e.y; r.px[6] = e.z; r.px[7] = e.w;
    } else {
#pragma unroll
      for (int k = 0; k < HIDE_PX; k++)
        if (k < r.valid) r.px[k >> 2] |= (uint32_t)src[k] << (8 * (k & 3));
    }
  }
  if (lmr && r.valid > 0) r.lbits = stream_bits32(d.map_bits, (uint32_t)((N + 31) >> 5), (uint32_t)p0);
}

__device__ __forceinline__ uint32_t zero_mask(const ImgDesc& d, const ChunkPx& r) {
  uint32_t z;
  if (d.variant != RDHEI_LMR) {
    // LSB == 0, pixel 4i+k -> bit 4i+k: the multiply gathers a word's four flags into
    // bits 28..31 (bit 8k -> 28+k), and the words are shifted in from the last one down
    z = 0;
#pragma unroll
    for (int i = 7; i >= 0; i--) z = __funnelshift_l(((~r.px[i]) & 0x01010101u) * 0x10204080u, z, 4);
  } else {
    z = ~r.lbits;
  }
  if (r.valid < 32) z &= r.valid <= 0 ? 0u : ((1u << r.valid) - 1u);
  return z;
}

__device__ __forceinline__ int slots_of(const ImgDesc& d, const rdhei_info* info) {
  const int b = d.b > 0 ? d.b : info->b;
  return d.variant == RDHEI_LMR ? b - 1 : b;
}

// PRMT selectors for the 4 pixels of a word with label-0 pattern z (bit q = pixel q):
//   expand:  byte q <- byte rank(q) of the consecutive fields (4 = zero byte) if z_q;
//   compact: byte j <- byte of the j-th label-0 pixel (4 = zero byte).
__host__ __device__ __forceinline__ uint32_t sel_expand(uint32_t z) {
  uint32_t sel = 0, r = 0;
  for (int q = 0; q < 4; q++) {
    const uint32_t nib = ((z >> q) & 1u) ? r++ : 4u;
    sel |= nib << (4 * q);
  }
  return sel;
}
__host__ __device__ __forceinline__ uint32_t sel_compact(uint32_t z) {
  uint32_t sel = 0x4444u, j = 0;
  for (int q = 0; q < 4; q++)
    if ((z >> q) & 1u) { sel = (sel & ~(0xFu << (4 * j))) | ((uint32_t)q << (4 * j)); j++; }
  return sel;
}

// The same with the fields in reversed byte order (first field in byte 3), which is
// the order the multiply-based field packing produces and consumes:
//   expand_rev:  byte q <- byte 3 - rank(q) if z_q, else the zero byte;
//   compact_rev: byte 3 - j <- byte of the j-th label-0 pixel, unused bytes zero.
__host__ __device__ __forceinline__ uint32_t sel_expand_rev(uint32_t z) {
  uint32_t sel = 0, r = 0;
  for (int q = 0; q < 4; q++) {
    const uint32_t nib = ((z >> q) & 1u) ? 3u - r++ : 4u;
    sel |= nib << (4 * q);
  }
  return sel;
}
__host__ __device__ __forceinline__ uint32_t sel_compact_rev(uint32_t z) {
  uint32_t sel = 0x4444u, j = 0;
  for (int q = 0; q < 4; q++)
    if ((z >> q) & 1u) { sel = (sel & ~(0xFu << (4 * (3 - j)))) | ((uint32_t)q << (4 * (3 - j))); j++; }
  return sel;
}
// Block-wide exclusive scan of one value per thread (256 threads); returns the
// exclusive prefix and the block total.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_tot, uint32_t& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  uint32_t base = 0, tot = 0;
#pragma unroll
  for (int i = 0; i < HIDE_THREADS / 32; i++) {
    const uint32_t u = warp_tot[i];
    base += i < warp ? u : 0u;
    tot += u;
  }
  __syncthreads();
  total = tot;
  return base + inc - v;
}


// 32 pixels from q0 of a raster range ending at qend (the run of a 64-row strip):
// pixel bytes from img (a coherent L2 load when `coherent`, i.e. when the calling
// kernel wrote them itself), and for LMR the packed map bits.
__device__ __forceinline__ void load_run(const ImgDesc& d, const uint8_t* img, uint64_t q0, uint64_t qend,
                                         bool coherent, ChunkPx& r) {
  r.valid = q0 < qend ? (int)umin64(HIDE_PX, qend - q0) : 0;
#pragma unroll
  for (int i = 0; i < 8; i++) r.px[i] = 0;
  r.lbits = 0xFFFFFFFFu;
  const uint8_t* src = img + q0;
  if (r.valid == HIDE_PX && ((reinterpret_cast<uintptr_t>(src) & 15) == 0)) {
    const uint4* s4 = reinterpret_cast<const uint4*>(src);
    const uint4 a = coherent ? __ldcg(s4) : __ldcs(s4), e = coherent ? __ldcg(s4 + 1) : __ldcs(s4 + 1);
    r.px[0] = a.x; r.px[1] = a.y; r.px[2] = a.z; r.px[3] = a.w;
    r.px[4] = e.x; r.px[5] = e.y; r.px[6] = e.z; r.px[7] = e.w;
  } else {
#pragma unroll
    for (int k = 0; k < HIDE_PX; k++)
      if (k < r.valid) r.px[k >> 2] |= (uint32_t)(coherent ? __ldcg(src + k) : src[k]) << (8 * (k & 3));
  }
  if (d.variant == RDHEI_LMR && r.valid > 0) {
    const uint64_t nw = ((uint64_t)d.H * d.W + 31) >> 5;
    r.lbits = coherent ? stream_bits32_cg(d.map_bits, (uint32_t)nw, (uint32_t)q0)
                       : stream_bits32(d.map_bits, (uint32_t)nw, (uint32_t)q0);
  }
}

// The same for 32 pixels at strip-relative offset q0 of a strip of n pixels whose first
// pixel is strip[0] (image pixel p0), in 32-bit offsets.  COHERENT: L2 loads (the fused
// encode reads back the strip it has just written), else streaming loads.
template <bool COHERENT = true>
__device__ __forceinline__ void load_strip_run(const ImgDesc& d, const uint8_t* strip, uint64_t p0, uint32_t q0,
                                               uint32_t n, ChunkPx& r) {
  r.valid = q0 < n ? (int)min((uint32_t)HIDE_PX, n - q0) : 0;
#pragma unroll
  for (int i = 0; i < 8; i++) r.px[i] = 0;
  r.lbits = 0xFFFFFFFFu;
  const uint8_t* src = strip + q0;
  if (r.valid == HIDE_PX && ((reinterpret_cast<uintptr_t>(src) & 15) == 0)) {
    const uint4* s4 = reinterpret_cast<const uint4*>(src);
    const uint4 a = COHERENT ? __ldcg(s4) : __ldcs(s4), e = COHERENT ? __ldcg(s4 + 1) : __ldcs(s4 + 1);
    r.px[0] = a.x; r.px[1] = a.y; r.px[2] = a.z; r.px[3] = a.w;
    r.px[4] = e.x; r.px[5] = e.y; r.px[6] = e.z; r.px[7] = e.w;
  } else {
#pragma unroll
    for (int k = 0; k < HIDE_PX; k++)
      if (k < r.valid) r.px[k >> 2] |= (uint32_t)(COHERENT ? __ldcg(src + k) : src[k]) << (8 * (k & 3));
  }
  if (d.variant == RDHEI_LMR && r.valid > 0) {
    const uint64_t nw = ((uint64_t)d.H * d.W + 31) >> 5;
    const uint32_t pos = (uint32_t)p0 + q0;
    r.lbits = COHERENT ? stream_bits32_cg(d.map_bits, (uint32_t)nw, pos) : stream_bits32(d.map_bits, (uint32_t)nw, pos);
  }
}

// Staging for the fused kernels' K2 keystream: enough 16-word ChaCha20 blocks for the
// message words of one chunk (at most 7 * 8192 bits) plus the two partial blocks at
// its ends.
constexpr int Z2BUF_WORDS = ((SBUF_WORDS + 15) / 16 + 2) * 16;

// Tables of byte-permute selectors, one entry per 4-pixel label-0 pattern.
struct SlotTables {
  uint32_t expand[16], expand_rev[16], compact_rev[16];
};
__device__ __forceinline__ void init_slot_tables(SlotTables& T) {
  const int t = threadIdx.x;
  if (t < 16) {
    T.expand[t] = sel_expand(t);
    T.expand_rev[t] = sel_expand_rev(t);
    T.compact_rev[t] = sel_compact_rev(t);
  }
}

// Hider: write message bits into the slots of my 32 pixels.  sbuf holds the
// K2-encrypted message as MSB-first words, its bit 0 being stream bit sb0 (a multiple of
// 32), and one zero word past the last one needed; my first slot is stream bit k0 and
// stream bits at or past E (the end of the message) are not written: those slots keep
// their pixel bits.
// POS is the type of the stream positions: 64-bit absolute ones, or 32-bit ones relative
// to a strip (the fused kernel), which cost fewer instructions.
template <typename POS>
__device__ __forceinline__ void spread_slots(uint32_t (&px)[8], uint32_t zmask, uint32_t slots, uint32_t fshift,
                                             const uint32_t* sbuf, POS sb0, POS k0, POS E,
                                             const SlotTables& T, uint32_t* err) {
  const uint32_t fmask = (1u << slots) - 1u;
  const uint32_t FREP = (fmask << fshift) * 0x01010101u;
  const uint32_t my_bits = (uint32_t)__popc(zmask) * slots;
  if (zmask && k0 + my_bits <= E) {
    // all my slots lie inside the message.  Per 4-pixel word: the next 32 stream
    // bits (left-aligned) hold the word's fields f0..f3 (first field most
    // significant); multiply-adds place f_k at bit fshift of byte 3 - k (the shifts
    // (3 - k)(8 - s) + fshift are all >= 0), one byte permute moves field r to the
    // r-th label-0 pixel, and a select writes the slot bits
    const uint32_t dsh = 8u - slots;
    const uint32_t m1 = fmask << slots, m2 = fmask << (2 * slots), m3 = fmask << (3 * slots);
    const uint32_t u0 = 1u << fshift, u1 = u0 << dsh, u2 = u1 << dsh, u3 = u2 << dsh;
    uint32_t idx = (uint32_t)(k0 - sb0);                            // stream position in sbuf
#pragma unroll
    for (int i = 0; i < 8; i++) {
      const uint32_t zw = (zmask >> (4 * i)) & 0xFu;
      const uint32_t w = idx >> 5;
      if (!RDHEI_IDX_OK(err, w + 1 < SBUF_WORDS)) break;
      const uint32_t Ew = __funnelshift_l(sbuf[w + 1], sbuf[w], idx & 31);
      const uint32_t F = Ew >> (32 - 4 * slots);                  // f0 .. f3, right-aligned
      const uint32_t cons = (F & fmask) * u0 + (F & m1) * u1 + (F & m2) * u2 + (F & m3) * u3;
      const uint32_t sel = T.expand_rev[zw];
      const uint32_t m = __byte_perm(FREP, 0, sel);                 // the field bits of the slot pixels
      px[i] = (px[i] & ~m) | __byte_perm(cons, 0, sel);
      idx += (uint32_t)__popc(zw) * slots;
    }
  } else if (zmask && k0 < E) {
    // the message ends inside my slots.  Per 4-pixel word: read the word's slots at
    // once, spread the fields to consecutive bytes, then move them to their pixels
    // with one byte permute; the slots past the message end keep their bits
    const uint32_t s2 = 2 * slots, s3 = 3 * slots;
    POS k = k0;
#pragma unroll
    for (int i = 0; i < 8; i++) {
      const uint32_t zw = (zmask >> (4 * i)) & 0xFu;
      const uint32_t nb = (uint32_t)__popc(zw) * slots;           // <= 28 bits
      if (nb && k < E && RDHEI_IDX_OK(err, ((k - sb0) >> 5) + 1 < SBUF_WORDS)) {
        const uint32_t avail = (POS)nb < E - k ? nb : (uint32_t)(E - k);
        const uint32_t Ew = get_bits(sbuf, (uint32_t)(k - sb0), avail) << (32 - avail);   // left-aligned
        const uint32_t rs = 32 - slots;
        const uint32_t cons = (Ew >> rs) | (((Ew << slots) >> rs) << 8) | (((Ew << s2) >> rs) << 16) |
                              (((Ew << s3) >> rs) << 24);
        const uint32_t zb = ((zw * 0x00204081u) & 0x01010101u) * 0xFFu;   // label-0 bytes
        uint32_t m = zb & FREP;
        if (avail < nb) {
          // the message ends inside this word: only its first `avail` slot bits
          uint32_t part = 0, left = avail;
          for (int j = 0; j < 4; j++) {
            const uint32_t n = left < slots ? left : slots;
            part |= (fmask & ~(fmask >> n)) << (8 * j);
            left -= n;
          }
          m &= __byte_perm(part << fshift, 0, T.expand[zw]);
        }
        px[i] = (px[i] & ~m) | (__byte_perm(cons << fshift, 0, T.expand[zw]) & m);
      }
      k += nb;
    }
  }
}

// Receiver: gather the slot fields of my 32 pixels into the chunk-local MSB-first
// stream sbuf at bit my_off.  Per 4-pixel word one byte permute puts the j-th label-0
// pixel in byte 3 - j; masked to the field bits, the fields are packed most-significant
// first by multiply-adds (byte j's field moves up by (4 - j)(8 - s) - fshift) and appended to a word
// that is stored once full: the words wholly inside my range are plain stores, the two
// I share with my neighbours are OR-ed (the caller cleared the range).
__device__ __forceinline__ void gather_slots(const uint32_t (&px)[8], uint32_t zmask, uint32_t slots,
                                             uint32_t fshift, uint32_t my_off, uint32_t* sbuf,
                                             const SlotTables& T, uint32_t* err) {
  const uint32_t FM = ((1u << slots) - 1u) << fshift;             // the field inside a byte
  const uint32_t dsh = 8u - slots;
  // byte j's field (at bit fshift) moves up by (4 - j)(8 - s) - fshift, which is >= 0
  // since fshift <= 8 - s: the field's offset inside its byte is folded into v0..v3
  const uint32_t v3 = (1u << dsh) >> fshift, v2 = v3 << dsh, v1 = v2 << dsh, v0 = v1 << dsh;
  uint32_t wi = my_off >> 5, c = my_off & 31, word = 0;
  bool first = true;
#pragma unroll
  for (int i = 0; i < 8; i++) {
    const uint32_t zw = (zmask >> (4 * i)) & 0xFu;
    const uint32_t nb = (uint32_t)__popc(zw) * slots;
    const uint32_t fld = __byte_perm(px[i], 0, T.compact_rev[zw]);
    const uint32_t P = (fld & FM) * v0 + (fld & (FM << 8)) * v1 + (fld & (FM << 16)) * v2 +
                       (fld & (FM << 24)) * v3;                  // nb bits, left-aligned
    word |= P >> c;
    c += nb;
    if (c >= 32) {
      if (RDHEI_IDX_OK(err, wi < SBUF_WORDS)) {
        if (first) atomicOr(sbuf + wi, word);
        else sbuf[wi] = word;
      }
      first = false;
      c -= 32;
      word = P << (nb - c);                                     // the bits that spilled over
      wi++;
    }
  }
  if (c && RDHEI_IDX_OK(err, wi < SBUF_WORDS)) atomicOr(sbuf + wi, word);
}

}  // namespace rdhei
