// hide.cu -- data hider (Sec. III-A-2, III-B-2) and K2 receiver (Sec. III-A-3,
// III-B-3): the payload slots of label-0 pixels, visited in raster order of the
// rotated image, hold the K2-encrypted message back to back.
//
// Both sides are split the way the paper describes them:
//   hider:    encrypt the message with K2 (e = m XOR z2, one ChaCha20 block per
//             thread over the message), then write e into the slots (k_scan);
//   receiver: concatenate the slots (k_scan), then decrypt with K2 (k_z2_xor).
// A pixel's first slot index is an exclusive prefix sum of slots over the raster.
// The scan is reduce-then-scan over chunks of 8192 pixels: the count pass counts each
// chunk's slots, k_offsets (one CTA per image) turns the counts into offsets, and
// k_scan writes (hider) or gathers (receiver) each chunk's slots at its offset.  The
// hider's encryption and count pass share one grid (k_z2_count); the receiver's count
// pass is k_count.  No CTA ever waits for another.
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
  if (lmr && r.valid > 0) r.lbits = stream_bits32(d.map_bits, (N + 31) >> 5, p0);
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
// 0xFF in the bytes of the label-0 pixels of pattern z
__host__ __device__ __forceinline__ uint32_t zero_bytes(uint32_t z) {
  return ((z & 1u) ? 0xFFu : 0u) | ((z & 2u) ? 0xFF00u : 0u) | ((z & 4u) ? 0xFF0000u : 0u) |
         ((z & 8u) ? 0xFF000000u : 0u);
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

// Pass 1 of the payload scan: slot count of every chunk, one warp per chunk.  Chunks
// are independent, so thousands of warps keep their reads in flight at once (no
// block-level synchronisation, no chunk-to-chunk dependency).  EMR counts the pixels
// whose LSB (the location-map bit) is 0, LMR the 0 bits of the packed map.
constexpr int COUNT_WARPS = 8;
__device__ __forceinline__ void count_chunks(const Batch& B, uint32_t cta) {
  pdl_wait();      // the previous kernel of the operation has finished
  pdl_trigger();
  const int lane = threadIdx.x & 31;
  const uint32_t g = cta * COUNT_WARPS + (threadIdx.x >> 5);
  if (g >= B.total_chunks) return;
  const int img = owner_of(B.chunk_prefix, B.n_images, g);
  const ImgDesc& d = B.desc[img];
  const rdhei_info* info = reinterpret_cast<const rdhei_info*>(d.info);
  const uint64_t N = (uint64_t)d.H * d.W;
  const uint64_t p0 = (uint64_t)(g - d.chunk_base) * SCAN_PX;
  const uint32_t valid = (uint32_t)umin64(SCAN_PX, N - p0);      // pixels of this chunk (>= 1)
  uint32_t z = 0;
  if (d.variant == RDHEI_LMR) {
    // SCAN_PX / 32 map words, MSB-first: pixel q of a word is bit 31 - q after the byte swap
    const uint32_t* mw = reinterpret_cast<const uint32_t*>(d.map_bits) + (p0 >> 5);
    const uint32_t nw = (valid + 31) >> 5;
#pragma unroll
    for (int k = 0; k < SCAN_PX / 32 / 32; k++) {
      const uint32_t w = (uint32_t)lane + 32u * k;
      if (w < nw) {
        uint32_t v = ~bswap32(__ldg(mw + w));
        const uint32_t left = valid - 32 * w;                      // pixels of this word inside the chunk
        if (left < 32) v &= ~0u << (32 - left);
        z += (uint32_t)__popc(v);
      }
    }
  } else {
    // pixel bytes: the 16-byte-aligned middle as uint4 (8 per lane in flight), the
    // head and tail bytes one per lane
    const uint8_t* src = d.src + p0;
    const uint32_t mis = (uint32_t)(reinterpret_cast<uintptr_t>(src) & 15);
    const uint32_t head = min(valid, (16u - mis) & 15u);
    const uint32_t nvec = (valid - head) >> 4;
    const uint32_t tail0 = head + 16 * nvec;
    if ((uint32_t)lane < head) z += (__ldg(src + lane) & 1u) ^ 1u;
    if ((uint32_t)lane < valid - tail0) z += (__ldg(src + tail0 + lane) & 1u) ^ 1u;
    const uint4* s4 = reinterpret_cast<const uint4*>(src + head);
    for (uint32_t k0 = 0; k0 < nvec; k0 += 32 * 8) {
      uint4 v[8];
#pragma unroll
      for (int j = 0; j < 8; j++) {
        const uint32_t k = k0 + lane + 32 * j;
        v[j] = k < nvec ? __ldcs(s4 + k) : make_uint4(~0u, ~0u, ~0u, ~0u);
      }
#pragma unroll
      for (int j = 0; j < 8; j++)
        z += (uint32_t)(__popc(~v[j].x & 0x01010101u) + __popc(~v[j].y & 0x01010101u) +
                        __popc(~v[j].z & 0x01010101u) + __popc(~v[j].w & 0x01010101u));
    }
  }
  z = __reduce_add_sync(0xffffffffu, z);
  if (lane == 0) reinterpret_cast<uint32_t*>(B.chunk_status)[g] = z * (uint32_t)slots_of(d, info);
}
__global__ void __launch_bounds__(32 * COUNT_WARPS) k_count(Batch B) { count_chunks(B, blockIdx.x); }

// Per image: exclusive prefix of the chunk counts (the bit offset at which each chunk's
// slots start -- Sec. III-A-2's "concatenation" order), the image totals and, for the
// extractor, clearing of the output words shared by two chunks.
template <bool EXTRACT>
__global__ void __launch_bounds__(HIDE_THREADS) k_offsets(Batch B) {
  pdl_wait();      // the previous kernel of the operation has finished
  pdl_trigger();
  __shared__ uint32_t warp_tot[HIDE_THREADS / 32];
  const int t = threadIdx.x;
  const int img = blockIdx.x;
  const ImgDesc& d = B.desc[img];
  rdhei_info* info = reinterpret_cast<rdhei_info*>(d.info);
  const uint32_t* cnt = reinterpret_cast<const uint32_t*>(B.chunk_status);
  uint32_t* off = reinterpret_cast<uint32_t*>(B.chunk_status) + B.total_chunks;
  const uint32_t base = d.chunk_base;
  const uint64_t lim_words = EXTRACT ? (d.max_bits + 31) >> 5 : 0;
  uint32_t* out = reinterpret_cast<uint32_t*>(d.bits_out);
  uint32_t running = 0;
  for (uint32_t c0 = 0; c0 < d.nchunks; c0 += HIDE_THREADS) {
    const uint32_t c = c0 + t;
    const uint32_t v = c < d.nchunks ? cnt[base + c] : 0u;
    uint32_t tot;
    const uint32_t ex = block_exclusive_scan(v, warp_tot, tot) + running;
    if (c < d.nchunks) {
      off[base + c] = ex;
      if (EXTRACT && v) {
        const uint64_t a = ex >> 5, e = (uint64_t)(ex + v) >> 5;
        if ((ex & 31) && a < lim_words) out[a] = 0u;                 // shared with the previous chunk
        if (((ex + v) & 31) && e < lim_words) out[e] = 0u;          // shared with the next chunk
      }
    }
    running += tot;
  }
  if (t == 0) {
    if (EXTRACT) {
      // the word holding the receiver's last requested bit may end inside a chunk
      const uint64_t E = umin64(d.max_bits, running);
      if ((E & 31) && (E >> 5) < lim_words) out[E >> 5] = 0u;
      info->extracted = E;
    } else {
      info->embedded = umin64(d.nbits, running);
      if (d.nbits > running) { info->status = ERR_CAPACITY; set_error(B.err, ERR_CAPACITY); }
    }
  }
}

// Pass 2 of the payload scan (persistent over a contiguous chunk range, next chunk
// prefetched).
// Hider: the K2-encrypted message bits of each chunk's slot range go into its slots,
// first bit into bit 7 (EMR) or 6 (LMR).  Receiver: the slots are concatenated; words
// inside the chunk's range are stored, words shared with a neighbour are OR-ed (they
// were cleared by k_offsets).
template <bool EXTRACT>
__global__ void __launch_bounds__(HIDE_THREADS, EXTRACT ? 5 : 4) k_scan(Batch B) {
  pdl_wait();      // the previous kernel of the operation has finished
  pdl_trigger();
  constexpr int EW = (SBUF_WORDS + HIDE_THREADS - 1) / HIDE_THREADS;   // message words per thread
  __shared__ uint32_t sbuf[SBUF_WORDS];   // hider: e words (MSB-first); receiver: raw slot stream
  __shared__ uint32_t warp_tot[HIDE_THREADS / 32];
  __shared__ uint32_t s_expand[16], s_expand_rev[16], s_compact_rev[16], s_zb[16];
  const int t = threadIdx.x;
  if (t < 16) {
    s_expand[t] = sel_expand(t);
    s_expand_rev[t] = sel_expand_rev(t);
    s_compact_rev[t] = sel_compact_rev(t);
    s_zb[t] = zero_bytes(t);
  }
  __syncthreads();
  const uint32_t* cnt = reinterpret_cast<const uint32_t*>(B.chunk_status);
  const uint32_t* off = cnt + B.total_chunks;
  // a contiguous range of chunks per CTA: the owning image only ever steps forward
  const uint32_t per = (B.total_chunks + gridDim.x - 1) / gridDim.x;
  uint32_t g = blockIdx.x * per;
  const uint32_t gend = (uint32_t)umin64((uint64_t)g + per, B.total_chunks);
  if (g >= gend) return;
  int img = owner_of(B.chunk_prefix, B.n_images, g);
  ChunkPx cur;
  issue_chunk(B.desc[img], g - B.desc[img].chunk_base, t, true, cur);
  uint64_t G = off[g];
  uint32_t T = cnt[g];
  while (g < gend) {
    const ImgDesc& d = B.desc[img];
    const rdhei_info* info = reinterpret_cast<const rdhei_info*>(d.info);
    const uint32_t slots = (uint32_t)slots_of(d, info);
    const uint32_t top = d.variant == RDHEI_LMR ? 6u : 7u;
    const uint32_t fshift = top + 1 - slots;
    const uint32_t fmask = (1u << slots) - 1u;
    const uint32_t c = g - d.chunk_base;
    const uint64_t p0 = (uint64_t)c * SCAN_PX + (uint64_t)HIDE_PX * t;

    // the message words of this chunk (hider), loads issued before the scan
    uint32_t ew[EW];
    uint64_t w_lo = G >> 5;
    uint32_t nw = 0;
    if (!EXTRACT) {
      const uint64_t end = umin64(G + T, d.nbits);
      nw = end > G ? (uint32_t)(((end - 1) >> 5) - w_lo + 1) : 0u;
      if (!RDHEI_IDX_OK(B.err, nw == 0 || (nw < SBUF_WORDS && w_lo + nw <= ((d.nbits + 31) >> 5)))) nw = 0;
      const uint32_t* e = reinterpret_cast<const uint32_t*>(d.ebuf) + w_lo;
#pragma unroll
      for (int i = 0; i < EW; i++) {
        const uint32_t k = t + i * HIDE_THREADS;
        ew[i] = k < nw ? __ldcs(e + k) : 0u;
      }
    }
    // next chunk in flight
    const uint32_t gn = g + 1;
    int imgn = img;
    ChunkPx nxt;
    uint64_t Gn = 0;
    uint32_t Tn = 0;
    if (gn < gend) {
      while (gn >= __ldg(B.chunk_prefix + imgn + 1)) imgn++;
      issue_chunk(B.desc[imgn], gn - B.desc[imgn].chunk_base, t, true, nxt);
      Gn = off[gn];
      Tn = cnt[gn];
    }

    const uint32_t zmask = zero_mask(d, cur);
    uint32_t Tb;
    const uint32_t my_off = block_exclusive_scan((uint32_t)__popc(zmask) * slots, warp_tot, Tb);

    if (!EXTRACT) {
#pragma unroll
      for (int i = 0; i < EW; i++) {
        const uint32_t k = t + i * HIDE_THREADS;
        if (k < nw) sbuf[k] = bswap32(ew[i]);
      }
      if (t == 0) sbuf[nw] = 0u;
      __syncthreads();
      const uint32_t FREP = (fmask << fshift) * 0x01010101u;
      const uint32_t my_bits = (uint32_t)__popc(zmask) * slots;
      if (zmask && G + my_off + my_bits <= d.nbits) {
        // all my slots lie inside the message.  Per 4-pixel word: the next 32 stream
        // bits (left-aligned) hold the word's fields f0..f3 (first field most
        // significant); multiply-adds place f_k at bit fshift of byte 3 - k (the shifts
        // (3 - k)(8 - s) + fshift are all >= 0), one byte permute moves field r to the
        // r-th label-0 pixel, and a select writes the slot bits
        const uint32_t dsh = 8u - slots;
        const uint32_t m1 = fmask << slots, m2 = fmask << (2 * slots), m3 = fmask << (3 * slots);
        const uint32_t u0 = 1u << fshift, u1 = u0 << dsh, u2 = u1 << dsh, u3 = u2 << dsh;
        uint32_t idx = (uint32_t)(G + my_off - 32 * w_lo);          // stream position in sbuf
#pragma unroll
        for (int i = 0; i < 8; i++) {
          const uint32_t zw = (zmask >> (4 * i)) & 0xFu;
          const uint32_t w = idx >> 5;
          if (!RDHEI_IDX_OK(B.err, w + 1 < SBUF_WORDS)) break;
          const uint32_t E = __funnelshift_l(sbuf[w + 1], sbuf[w], idx & 31);
          const uint32_t F = E >> (32 - 4 * slots);                 // f0 .. f3, right-aligned
          const uint32_t cons = (F & fmask) * u0 + (F & m1) * u1 + (F & m2) * u2 + (F & m3) * u3;
          const uint32_t m = s_zb[zw] & FREP;
          cur.px[i] = (cur.px[i] & ~m) | __byte_perm(cons, 0, s_expand_rev[zw]);
          idx += (uint32_t)__popc(zw) * slots;
        }
      } else if (zmask && G + my_off < d.nbits) {
        // the message ends inside my slots.  Per 4-pixel word: read the word's slots at
        // once, spread the fields to consecutive bytes, then move them to their pixels
        // with one byte permute; the slots past the message end keep their bits
        const uint64_t base = 32 * w_lo;
        const uint32_t s2 = 2 * slots, s3 = 3 * slots;
        uint64_t k = G + my_off;
#pragma unroll
        for (int i = 0; i < 8; i++) {
          const uint32_t zw = (zmask >> (4 * i)) & 0xFu;
          const uint32_t nb = (uint32_t)__popc(zw) * slots;         // <= 28 bits
          if (nb && k < d.nbits && RDHEI_IDX_OK(B.err, ((k - base) >> 5) + 1 < SBUF_WORDS)) {
            const uint32_t avail = (uint32_t)umin64(nb, d.nbits - k);
            const uint32_t E = get_bits(sbuf, (uint32_t)(k - base), avail) << (32 - avail);   // left-aligned
            const uint32_t rs = 32 - slots;
            const uint32_t cons = (E >> rs) | (((E << slots) >> rs) << 8) | (((E << s2) >> rs) << 16) |
                                  (((E << s3) >> rs) << 24);
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
              m &= __byte_perm(part << fshift, 0, s_expand[zw]);
            }
            cur.px[i] = (cur.px[i] & ~m) | (__byte_perm(cons << fshift, 0, s_expand[zw]) & m);
          }
          k += nb;
        }
      }
      uint8_t* dst = d.dst + p0;
      if (cur.valid == HIDE_PX && ((reinterpret_cast<uintptr_t>(dst) & 15) == 0)) {
        __stcs(reinterpret_cast<uint4*>(dst), make_uint4(cur.px[0], cur.px[1], cur.px[2], cur.px[3]));
        __stcs(reinterpret_cast<uint4*>(dst) + 1, make_uint4(cur.px[4], cur.px[5], cur.px[6], cur.px[7]));
      } else {
#pragma unroll
        for (int k = 0; k < HIDE_PX; k++)
          if (k < cur.valid) dst[k] = (uint8_t)(cur.px[k >> 2] >> (8 * (k & 3)));
      }
    } else {
      for (int i = t; i < (int)((Tb >> 5) + 2) && i < SBUF_WORDS; i += HIDE_THREADS) sbuf[i] = 0u;
      __syncthreads();
      // gather my slots into the chunk-local stream.  Per 4-pixel word one byte permute
      // puts the j-th label-0 pixel in byte 3 - j; masked to the field bits, the fields
      // are packed most-significant first by multiply-adds (byte j moves up by
      // (4 - j)(8 - s)) and appended to a word that is stored once full: the words
      // wholly inside my range are plain stores, the two I share with my neighbours are
      // OR-ed (the range was cleared above)
      {
        const uint32_t FREP = fmask * 0x01010101u;
        const uint32_t dsh = 8u - slots;
        const uint32_t v3 = 1u << dsh, v2 = v3 << dsh, v1 = v2 << dsh, v0 = v1 << dsh;
        uint32_t wi = my_off >> 5, c = my_off & 31, word = 0;
        bool first = true;
#pragma unroll
        for (int i = 0; i < 8; i++) {
          const uint32_t zw = (zmask >> (4 * i)) & 0xFu;
          const uint32_t nb = (uint32_t)__popc(zw) * slots;
          const uint32_t fld = (__byte_perm(cur.px[i], 0, s_compact_rev[zw]) >> fshift) & FREP;
          const uint32_t P = (fld & 0xFFu) * v0 + (fld & 0xFF00u) * v1 + (fld & 0xFF0000u) * v2 +
                             (fld & 0xFF000000u) * v3;                 // nb bits, left-aligned
          word |= P >> c;
          c += nb;
          if (c >= 32) {
            if (RDHEI_IDX_OK(B.err, wi < SBUF_WORDS)) {
              if (first) atomicOr(sbuf + wi, word);
              else sbuf[wi] = word;
            }
            first = false;
            c -= 32;
            word = P << (nb - c);                                     // the bits that spilled over
            wi++;
          }
        }
        if (c && RDHEI_IDX_OK(B.err, wi < SBUF_WORDS)) atomicOr(sbuf + wi, word);
      }
      __syncthreads();
      // words of [G, min(G + T, E)), E = bits the receiver asked for and the image holds
      const uint64_t E = info->extracted;
      const uint64_t end = umin64(G + T, E);
      uint32_t* out = reinterpret_cast<uint32_t*>(d.bits_out);
      if (end > G) {
        const uint64_t w_hi = (end - 1) >> 5;
        for (uint64_t w = w_lo + t; w <= w_hi; w += HIDE_THREADS) {
          const uint64_t b0 = 32 * w;
          const uint64_t lo = b0 > G ? b0 : G, hi = b0 + 32 < end ? b0 + 32 : end;   // my bits of word w
          if (!RDHEI_IDX_OK(B.err, w < ((d.max_bits + 31) >> 5) && ((lo - G) >> 5) + 1 < SBUF_WORDS)) continue;
          uint32_t raw = get_bits(sbuf, (uint32_t)(lo - G), (uint32_t)(hi - lo));
          raw <<= (uint32_t)(b0 + 32 - hi);
          if (lo == b0 && hi == b0 + 32) out[w] = bswap32(raw);
          else atomicOr(out + w, bswap32(raw));
        }
      }
    }
    __syncthreads();   // sbuf is rewritten by the next chunk
    g = gn;
    img = imgn;
    cur = nxt;
    G = Gn;
    T = Tn;
  }
}

// K2 keystream over a message: one ChaCha20 block (512 message bits) per thread.
//   encrypt (hider):     e[w] = m[w] XOR z2[w] into the workspace e buffer;
//   decrypt (receiver):  out[w] ^= z2[w] for the extracted bits, zero past `extracted`.
// Words are the stream's bytes read little-endian, so the XOR is byte-wise.
template <bool DECRYPT>
__device__ __forceinline__ void z2_block(const Batch& B, uint32_t j) {   // j: global block index
  if (j >= B.total_z2_blocks) return;
  const int img = owner_of(B.z2_prefix, B.n_images, j);
  const ImgDesc& d = B.desc[img];
  const rdhei_info* info = reinterpret_cast<const rdhei_info*>(d.info);
  const uint32_t blk = j - __ldg(B.z2_prefix + img);
  // the keystream block needs nothing that an earlier kernel writes: it is computed
  // while the previous kernel finishes; the bit count and the message are read after
  // the wait
  uint32_t o[16];
  chacha20_block(d.k2, blk, d.n2, o, d.one);
  pdl_wait();
  pdl_trigger();
  const uint64_t nbits = DECRYPT ? info->extracted : d.nbits;
  const uint64_t nwords = (nbits + 31) >> 5;
  const uint64_t w0 = (uint64_t)blk * 16;
  if (w0 >= nwords) return;
  const uint32_t* in = reinterpret_cast<const uint32_t*>(DECRYPT ? d.bits_out : d.payload);
  uint32_t* out = reinterpret_cast<uint32_t*>(DECRYPT ? d.bits_out : d.ebuf);
  const int nw = (int)umin64(16, nwords - w0);
  if (nw == 16 && ((reinterpret_cast<uintptr_t>(in + w0) & 15) == 0) &&
      ((reinterpret_cast<uintptr_t>(out + w0) & 15) == 0)) {
    const uint4* i4 = reinterpret_cast<const uint4*>(in + w0);
    uint4* o4 = reinterpret_cast<uint4*>(out + w0);
#pragma unroll
    for (int q = 0; q < 4; q++) {
      uint4 v = i4[q];
      v.x ^= o[4 * q]; v.y ^= o[4 * q + 1]; v.z ^= o[4 * q + 2]; v.w ^= o[4 * q + 3];
      o4[q] = v;
    }
  } else {
#pragma unroll
    for (int k = 0; k < 16; k++)
      if (k < nw) out[w0 + k] = in[w0 + k] ^ o[k];
  }
  if (DECRYPT && w0 + nw == nwords && (nbits & 31)) {
    // the last word holds bits past the message: keep them zero
    const uint32_t keep = (uint32_t)(nbits & 31);
    out[nwords - 1] &= bswap32(0xFFFFFFFFu << (32 - keep));
  }
}
template <bool DECRYPT>
__global__ void __launch_bounds__(128) k_z2_xor(Batch B) { z2_block<DECRYPT>(B, blockIdx.x * blockDim.x + threadIdx.x); }

// The hider's first kernel: the K2 encryption of the message and the slot count of
// every chunk, in one grid.  The two are independent of each other; the count is
// bound by its reads of the image and the encryption by ChaCha20's integer work, so
// their CTAs alternate (even blocks count, odd blocks encrypt, while both have work
// left) and share the SMs instead of running one after the other.
constexpr int Z2C_THREADS = 32 * COUNT_WARPS;
__global__ void __launch_bounds__(Z2C_THREADS) k_z2_count(Batch B, uint32_t count_ctas, uint32_t z2_ctas) {
  const uint32_t both = 2 * min(count_ctas, z2_ctas), b = blockIdx.x;
  const bool count = b < both ? (b & 1u) == 0 : count_ctas > z2_ctas;
  const uint32_t i = b < both ? b >> 1 : b - both / 2;
  if (count) count_chunks(B, i);
  else z2_block<false>(B, i * Z2C_THREADS + threadIdx.x);
}

// LMR side information into bit 7 (Sec. III-B-1): pixel q < side_nbits.
__global__ void k_lmr_side(Batch B) {
  pdl_wait();      // the previous kernel of the operation has finished
  pdl_trigger();
  const uint32_t g = blockIdx.x;
  const int img = owner_of(B.chunk_prefix, B.n_images, g);
  const ImgDesc& d = B.desc[img];
  const uint64_t N = (uint64_t)d.H * d.W;
  const uint64_t p0 = (uint64_t)(g - d.chunk_base) * CHUNK_PX + (uint64_t)HIDE_PX * threadIdx.x;
  if (p0 >= N || p0 >= d.side_nbits || !d.side_bits) return;
  const int n = (int)umin64(umin64(HIDE_PX, N - p0), d.side_nbits - p0);
  const uint32_t sb = stream_bits32(d.side_bits, (d.side_nbits + 31) >> 5, p0);
  for (int k = 0; k < n; k++) d.dst[p0 + k] = (uint8_t)((d.dst[p0 + k] & 0x7Fu) | (((sb >> k) & 1u) << 7));
}

// one resident wave of a persistent kernel (CTAs per SM from the occupancy calculator)
template <typename K>
static int persistent_grid(K kernel, uint32_t work) {
  int dev = 0, sms = 1, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, HIDE_THREADS, 0);
  const uint32_t g = (uint32_t)(sms > 0 ? sms : 1) * (uint32_t)(per_sm > 0 ? per_sm : 1);
  return (int)(work < g ? work : g);
}
// count + per-image offsets
void launch_offsets(const Batch& B, bool extract, cudaStream_t st);
void launch_count(const Batch& B, bool extract, cudaStream_t st) {
  if (B.total_chunks == 0) return;
  launch_pdl(k_count, dim3((B.total_chunks + COUNT_WARPS - 1) / COUNT_WARPS), dim3(32 * COUNT_WARPS), 0, st, B);
  launch_offsets(B, extract, st);
}
void launch_offsets(const Batch& B, bool extract, cudaStream_t st) {
  if (B.total_chunks == 0) return;
  if (extract) launch_pdl(k_offsets<true>, dim3(B.n_images), dim3(HIDE_THREADS), 0, st, B);
  else launch_pdl(k_offsets<false>, dim3(B.n_images), dim3(HIDE_THREADS), 0, st, B);
}
// hider: message encryption and slot counts in one grid (the offsets follow)
void launch_z2_count(const Batch& B, cudaStream_t st) {
  const uint32_t cc = (B.total_chunks + COUNT_WARPS - 1) / COUNT_WARPS;
  const uint32_t zc = (B.total_z2_blocks + Z2C_THREADS - 1) / Z2C_THREADS;
  if (cc + zc == 0) return;
  launch_pdl(k_z2_count, dim3(cc + zc), dim3(Z2C_THREADS), 0, st, B, cc, zc);
}
void launch_scan(const Batch& B, bool extract, cudaStream_t st) {
  if (B.total_chunks == 0) return;
  if (extract) launch_pdl(k_scan<true>, dim3(persistent_grid(k_scan<true>, B.total_chunks)), dim3(HIDE_THREADS), 0, st, B);
  else launch_pdl(k_scan<false>, dim3(persistent_grid(k_scan<false>, B.total_chunks)), dim3(HIDE_THREADS), 0, st, B);
}
void launch_z2_xor(const Batch& B, bool decrypt, cudaStream_t st) {
  if (B.total_z2_blocks == 0) return;
  const uint32_t grid = (B.total_z2_blocks + 127) / 128;
  if (decrypt) launch_pdl(k_z2_xor<true>, dim3(grid), dim3(128), 0, st, B);
  else launch_pdl(k_z2_xor<false>, dim3(grid), dim3(128), 0, st, B);
}
void launch_lmr_side(const Batch& B, cudaStream_t st) {
  if (B.total_chunks == 0) return;
  launch_pdl(k_lmr_side, dim3(B.total_chunks), dim3(HIDE_THREADS), 0, st, B);
}

}  // namespace rdhei
