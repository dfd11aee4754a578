// hide.cu -- data hider (Sec. III-A-2, III-B-2) and K2 receiver (Sec. III-A-3,
// III-B-3): the payload slots of label-0 pixels, visited in raster order of the
// rotated image, hold the K2-encrypted message back to back.
//
// Both sides are split the way the paper describes them:
//   hider:    encrypt the message with K2 (k_z2_xor: e = m XOR z2, one ChaCha20 block
//             per thread over the message), then write e into the slots (k_scan);
//   receiver: concatenate the slots (k_scan), then decrypt with K2 (k_z2_xor).
// A pixel's first slot index is an exclusive prefix sum of slots over the raster.
// Chunks of 8192 pixels are taken in ticket order; each scans its own pixels
// (warp shuffles), publishes its slot count, then finds its offset with a decoupled
// look-back over up to 32 predecessors per step.  The status word of a chunk packs a
// flag (2 bits), a 30-bit count or inclusive prefix, and the last 32 raw stream bits
// up to that point, which the extractor uses to complete the 32-bit word it shares
// with earlier chunks.
#include "common.cuh"
#include "../../include/rdhei.h"

namespace rdhei {

constexpr int TK_HIDE = 1;
constexpr int HIDE_THREADS = 256;
constexpr int HIDE_PX = 32;                          // pixels per thread
constexpr int SCAN_PX = HIDE_THREADS * HIDE_PX;      // 8192 pixels per chunk
static_assert(SCAN_PX == CHUNK_PX, "chunk size shared with the host layout");
constexpr int SBUF_WORDS = 7 * SCAN_PX / 32 + 4;     // slots of one chunk, in 32-bit words

__device__ __forceinline__ unsigned long long pack_status(uint32_t flag, uint32_t value, uint32_t tail) {
  return ((unsigned long long)flag << 62) | ((unsigned long long)(value & 0x3FFFFFFFu) << 32) | tail;
}

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

// Decoupled look-back by one warp: the exclusive slot offset G of chunk g and the last
// 32 raw stream bits before it.  Publishes the chunk's aggregate first, its inclusive
// value after.  Image chunk 0 is inclusive at once.
template <bool EXTRACT>
__device__ __forceinline__ void lookback(const Batch& B, const ImgDesc& d, rdhei_info* info, uint32_t g, uint32_t c,
                                         uint32_t T, uint32_t tail, uint32_t& G_out, uint32_t& carry_out) {
  const int lane = threadIdx.x & 31;
  unsigned long long* st = B.chunk_status + g;
  uint32_t G = 0, acc = 0;
  if (c == 0) {
    if (lane == 0) st_release_u64(st, pack_status(2, T, tail));
  } else {
    if (lane == 0) st_release_u64(st, pack_status(1, T, tail));
    uint32_t have = 0;
    int64_t cur = (int64_t)g - 1;
    const int64_t first = (int64_t)d.chunk_base;
    const uint64_t t0 = globaltimer_ns();
    while (true) {
      const int64_t idx = cur - lane;
      unsigned long long sw = 0;
      bool late = false;
      if (idx >= first) {
        while (true) {
          sw = ld_acquire_u64(B.chunk_status + idx);
          if ((sw >> 62) != 0) break;
          if (globaltimer_ns() - t0 > WAIT_LIMIT_NS) { late = true; break; }
          __nanosleep(32);
        }
      }
      if (__any_sync(0xffffffffu, late)) {
        if (lane == 0) { set_error(B.err, ERR_TIMEOUT); info->status = ERR_TIMEOUT; }
        break;
      }
      const uint32_t f = idx >= first ? (uint32_t)(sw >> 62) : 2u;
      const uint32_t incm = __ballot_sync(0xffffffffu, f == 2);
      const int L = incm ? __ffs(incm) - 1 : 31;       // lanes 0..L follow the nearest inclusive one
      const uint32_t v = lane <= L ? ((uint32_t)(sw >> 32) & 0x3FFFFFFFu) : 0u;
      uint32_t sum = v;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
      G += sum;
      if (EXTRACT) {
        const uint32_t tl = (uint32_t)sw;
        for (int j = 0; j <= L && have < 32; j++) {
          const uint32_t vj = __shfl_sync(0xffffffffu, v, j), tj = __shfl_sync(0xffffffffu, tl, j);
          const uint32_t fj = __shfl_sync(0xffffffffu, f, j);
          if (fj == 2) {
            acc |= have == 0 ? tj : (tj << have);
            have = 32;
          } else if (vj) {
            const uint32_t nb = vj < 32 ? vj : 32;
            const uint32_t part = nb == 32 ? tj : (tj & ((1u << nb) - 1u));
            acc |= have == 0 ? part : (part << have);
            have = have + vj > 32 ? 32 : have + vj;
          }
        }
      }
      if (incm) break;
      cur -= 32;
    }
    uint32_t itail = 0;
    if (EXTRACT) itail = T >= 32 ? tail : (T > 0 ? ((acc << T) | tail) : acc);
    if (lane == 0) st_release_u64(st, pack_status(2, G + T, itail));
  }
  G_out = G;
  carry_out = acc;
}

template <bool EXTRACT>
__global__ void __launch_bounds__(HIDE_THREADS) k_scan(Batch B) {
  __shared__ uint32_t sbuf[SBUF_WORDS];   // embed: e words of the chunk (MSB-first); extract: raw stream
  __shared__ uint32_t warp_tot[HIDE_THREADS / 32];
  __shared__ uint32_t s_ticket, s_G, s_carry;

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if (t == 0) s_ticket = atomicAdd(B.tickets + TK_HIDE, 1u);
  if (EXTRACT)
    for (int i = t; i < SBUF_WORDS; i += HIDE_THREADS) sbuf[i] = 0u;
  __syncthreads();
  const uint32_t g = s_ticket;
  const int img = owner_of(B.chunk_prefix, B.n_images, g);
  const ImgDesc& d = B.desc[img];
  rdhei_info* info = reinterpret_cast<rdhei_info*>(d.info);
  const uint64_t N = (uint64_t)d.H * d.W;
  const uint32_t c = g - d.chunk_base;
  const int b = d.b > 0 ? d.b : info->b;
  const bool lmr = d.variant == RDHEI_LMR;
  const uint32_t slots = lmr ? (uint32_t)(b - 1) : (uint32_t)b;
  const uint32_t top = lmr ? 6u : 7u;
  const uint32_t fshift = top + 1 - slots;                    // field's lowest bit position

  // ---- my 32 pixels, their labels and slot count -----------------------------------
  const uint64_t p0 = (uint64_t)c * SCAN_PX + (uint64_t)HIDE_PX * t;
  const int valid = p0 < N ? (int)umin64(HIDE_PX, N - p0) : 0;
  const uint8_t* src = d.src + p0;
  uint32_t px[8];
#pragma unroll
  for (int i = 0; i < 8; i++) px[i] = 0;
  if (valid == HIDE_PX && ((reinterpret_cast<uintptr_t>(src) & 15) == 0)) {
    const uint4 a = *reinterpret_cast<const uint4*>(src), e = *reinterpret_cast<const uint4*>(src + 16);
    px[0] = a.x; px[1] = a.y; px[2] = a.z; px[3] = a.w; px[4] = e.x; px[5] = e.y; px[6] = e.z; px[7] = e.w;
  } else {
    for (int k = 0; k < valid; k++) px[k >> 2] |= (uint32_t)src[k] << (8 * (k & 3));
  }
  uint32_t zmask;   // bit k: pixel k is redundant (label 0)
  if (!lmr) {
    zmask = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) {
      const uint32_t nib = (((~px[i]) & 0x01010101u) * 0x01020408u) >> 24;   // LSB == 0, pixel 4i+k -> bit k
      zmask |= (nib & 0xFu) << (4 * i);
    }
  } else {
    zmask = ~stream_bits32(d.map_bits, (N + 31) >> 5, p0);
  }
  if (valid < 32) zmask &= valid <= 0 ? 0u : ((1u << valid) - 1u);
  const uint32_t mycnt = (uint32_t)__popc(zmask) * slots;

  // ---- block scan ------------------------------------------------------------------------
  uint32_t inc = mycnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  uint32_t wbase = 0, T = 0;
#pragma unroll
  for (int i = 0; i < HIDE_THREADS / 32; i++) {
    const uint32_t v = warp_tot[i];
    wbase += i < warp ? v : 0u;
    T += v;
  }
  const uint32_t my_off = wbase + inc - mycnt;            // exclusive, local to the chunk

  if (EXTRACT) {
    // gather my slots into the chunk-local raw stream (32 bits at a time)
    uint64_t acc = 0;
    uint32_t nacc = 0, o = my_off;
    uint32_t zm = zmask;
    while (zm) {
      const int k = __ffs(zm) - 1;
      zm &= zm - 1;
      const uint32_t field = (px[k >> 2] >> (8 * (k & 3) + fshift)) & ((1u << slots) - 1u);
      acc = (acc << slots) | field;
      nacc += slots;
      if (nacc >= 32) {
        nacc -= 32;
        or_bits(sbuf, o, (uint32_t)(acc >> nacc), 32);
        o += 32;
      }
    }
    if (nacc) or_bits(sbuf, o, (uint32_t)acc & ((1u << nacc) - 1u), nacc);
    __syncthreads();
  }

  // ---- offset of the chunk ---------------------------------------------------------------
  if (warp == 0) {
    uint32_t tail = 0;
    if (EXTRACT && T > 0) tail = T >= 32 ? get_bits(sbuf, T - 32, 32) : get_bits(sbuf, 0, T);
    uint32_t G, carry;
    lookback<EXTRACT>(B, d, info, g, c, T, tail, G, carry);
    if (lane == 0) { s_G = G; s_carry = carry; }
  }
  __syncthreads();
  const uint64_t G = s_G, Gend = G + T;
  const bool last = c + 1 == d.nchunks;
  if (last && t == 0) {
    if (EXTRACT) {
      info->extracted = umin64(d.max_bits, Gend);
    } else {
      info->embedded = umin64(d.nbits, Gend);
      if (d.nbits > Gend) { info->status = ERR_CAPACITY; set_error(B.err, ERR_CAPACITY); }
    }
  }

  if (!EXTRACT) {
    // the K2-encrypted message words covering [G, min(Gend, nbits)), MSB-first
    const uint64_t end = umin64(Gend, d.nbits);
    const uint32_t* ew = reinterpret_cast<const uint32_t*>(d.ebuf);
    const uint64_t w_lo = G >> 5;
    const uint32_t nw = end > G ? (uint32_t)(((end - 1) >> 5) - w_lo + 1) : 0u;
    for (uint32_t i = t; i < nw; i += HIDE_THREADS) sbuf[i] = bswap32(ew[w_lo + i]);
    if (t == 0) sbuf[nw] = 0u;
    __syncthreads();
    if (zmask && G + my_off < d.nbits) {
      uint64_t k = G + my_off;
      const uint64_t base = 32 * w_lo;
      uint32_t zm = zmask;
      while (zm && k < d.nbits) {
        const int q = __ffs(zm) - 1;
        zm &= zm - 1;
        const uint32_t n = (uint32_t)umin64(slots, d.nbits - k);
        const uint32_t e = get_bits(sbuf, (uint32_t)(k - base), n);
        const uint32_t bs = 8 * (q & 3) + (top + 1 - n);        // first bit into bit `top`
        const uint32_t m = ((1u << n) - 1u) << bs;
        px[q >> 2] = (px[q >> 2] & ~m) | (e << bs);
        k += slots;
      }
    }
    uint8_t* dst = d.dst + p0;
    if (valid == HIDE_PX && ((reinterpret_cast<uintptr_t>(dst) & 15) == 0)) {
      reinterpret_cast<uint4*>(dst)[0] = make_uint4(px[0], px[1], px[2], px[3]);
      reinterpret_cast<uint4*>(dst)[1] = make_uint4(px[4], px[5], px[6], px[7]);
    } else {
      for (int k = 0; k < valid; k++) dst[k] = (uint8_t)(px[k >> 2] >> (8 * (k & 3)));
    }
  } else {
    // raw output words whose last bit lies in this chunk (the image's last chunk also
    // writes the final partial word), zero past min(max_bits, Gend)
    const uint64_t limit = umin64(d.max_bits, Gend);
    const uint64_t w_lo = G >> 5;
    uint64_t hi_excl = Gend >> 5;
    if (last && (Gend & 31)) hi_excl += 1;
    const uint64_t lim = (d.max_bits + 31) >> 5;
    if (hi_excl > lim) hi_excl = lim;
    uint32_t* out = reinterpret_cast<uint32_t*>(d.bits_out);
    const uint32_t carry = s_carry;
    for (uint64_t w = w_lo + t; w < hi_excl; w += HIDE_THREADS) {
      const uint64_t b0 = 32 * w;
      uint32_t raw;
      if (b0 >= G) {
        raw = get_bits(sbuf, (uint32_t)(b0 - G), 32);
      } else {
        const uint32_t k = (uint32_t)(G - b0);             // 1..31 bits from earlier chunks
        raw = ((carry & ((1u << k) - 1u)) << (32 - k)) | (sbuf[0] >> k);
      }
      if (b0 + 32 > limit) {
        const uint64_t keep = limit > b0 ? limit - b0 : 0;
        raw = keep == 0 ? 0u : (raw & (0xFFFFFFFFu << (32 - keep)));
      }
      out[w] = bswap32(raw);
    }
  }
}

// K2 keystream over a message: one ChaCha20 block (512 message bits) per thread.
//   encrypt (hider):     e[w] = m[w] XOR z2[w] into the workspace e buffer;
//   decrypt (receiver):  out[w] ^= z2[w] for the extracted bits, zero past `extracted`.
// Words are the stream's bytes read little-endian, so the XOR is byte-wise.
template <bool DECRYPT>
__global__ void __launch_bounds__(128) k_z2_xor(Batch B) {
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;   // global block index
  if (j >= B.total_z2_blocks) return;
  const int img = owner_of(B.z2_prefix, B.n_images, j);
  const ImgDesc& d = B.desc[img];
  const rdhei_info* info = reinterpret_cast<const rdhei_info*>(d.info);
  const uint32_t blk = j - __ldg(B.z2_prefix + img);
  const uint64_t nbits = DECRYPT ? info->extracted : d.nbits;
  const uint64_t nwords = (nbits + 31) >> 5;
  const uint64_t w0 = (uint64_t)blk * 16;
  if (w0 >= nwords) return;
  uint32_t o[16];
  chacha20_block(d.k2, blk, d.n2, o);
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

// LMR side information into bit 7 (Sec. III-B-1): pixel q < side_nbits.
__global__ void k_lmr_side(Batch B) {
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

void launch_scan(const Batch& B, bool extract, cudaStream_t st) {
  if (B.total_chunks == 0) return;
  if (extract) k_scan<true><<<B.total_chunks, HIDE_THREADS, 0, st>>>(B);
  else k_scan<false><<<B.total_chunks, HIDE_THREADS, 0, st>>>(B);
}
void launch_z2_xor(const Batch& B, bool decrypt, cudaStream_t st) {
  if (B.total_z2_blocks == 0) return;
  const uint32_t grid = (B.total_z2_blocks + 127) / 128;
  if (decrypt) k_z2_xor<true><<<grid, 128, 0, st>>>(B);
  else k_z2_xor<false><<<grid, 128, 0, st>>>(B);
}
void launch_lmr_side(const Batch& B, cudaStream_t st) {
  if (B.total_chunks == 0) return;
  k_lmr_side<<<B.total_chunks, HIDE_THREADS, 0, st>>>(B);
}

}  // namespace rdhei
