// hide.cu -- data hider (Sec. III-A-2, III-B-2) and K2 receiver (Sec. III-A-3,
// III-B-3): the payload slots of label-0 pixels, visited in raster order of the
// rotated image, hold the K2-encrypted message back to back.
//
// A pixel's first slot index is an exclusive prefix sum of slots over the raster.
// Chunks of 4096 pixels are taken in ticket order; each scans its own pixels (warp
// shuffles), publishes its slot count, then finds its offset with a decoupled
// look-back.  The status word of a chunk packs flag (2 bits), a 30-bit count or
// inclusive prefix, and the last 32 raw stream bits up to that point, which the
// extractor uses to complete the 32-bit word it shares with earlier chunks.
#include "common.cuh"
#include "../../include/rdhei.h"

namespace rdhei {

constexpr int TK_HIDE = 1;
constexpr int HIDE_THREADS = 256;
constexpr int EBUF_WORDS = 7 * CHUNK_PX / 32 + 48;    // slots of one chunk + block alignment

__device__ __forceinline__ unsigned long long pack_status(uint32_t flag, uint32_t value, uint32_t tail) {
  return ((unsigned long long)flag << 62) | ((unsigned long long)(value & 0x3FFFFFFFu) << 32) | tail;
}

// n (<= 32) bits of an MSB-first word array starting at bit idx, MSB-first in the result's low n bits
__device__ __forceinline__ uint32_t get_bits(const uint32_t* buf, uint32_t idx, uint32_t n) {
  if (n == 0) return 0u;
  const uint32_t w = idx >> 5, sh = idx & 31;
  uint64_t v = ((uint64_t)buf[w] << 32) | buf[w + 1];
  return (uint32_t)((v << sh) >> (64 - n));
}
// OR n (<= 32) bits (value's low n bits, MSB-first) into an MSB-first shared word array
__device__ __forceinline__ void or_bits(uint32_t* buf, uint32_t idx, uint32_t val, uint32_t n) {
  if (n == 0) return;
  const uint32_t w = idx >> 5, sh = idx & 31;
  const uint64_t run = (((uint64_t)val) << (64 - n)) >> sh;
  const uint32_t hi = (uint32_t)(run >> 32), lo = (uint32_t)run;
  if (hi) atomicOr(buf + w, hi);
  if (lo) atomicOr(buf + w + 1, lo);
}

template <bool EXTRACT>
__global__ void __launch_bounds__(HIDE_THREADS) k_hide(Batch B) {
  __shared__ uint32_t ebuf[EBUF_WORDS];         // embed: z2 ^ payload; extract: z2
  __shared__ uint32_t lbuf[EXTRACT ? EBUF_WORDS : 1];   // extract: the chunk's raw stream
  __shared__ uint32_t warp_tot[HIDE_THREADS / 32];
  __shared__ uint32_t s_ticket, s_G, s_carry, s_T;

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if (t == 0) s_ticket = atomicAdd(B.tickets + TK_HIDE, 1u);
  __syncthreads();
  const uint32_t g = s_ticket;
  const int img = owner_of(B.chunk_prefix, B.n_images, g);
  const ImgDesc& d = B.desc[img];
  rdhei_info* info = reinterpret_cast<rdhei_info*>(d.info);
  const uint64_t N = (uint64_t)d.H * d.W;
  const uint32_t c = g - d.chunk_base;
  const uint64_t start = (uint64_t)c * CHUNK_PX;
  const int b = d.b > 0 ? d.b : info->b;
  const bool lmr = d.variant == RDHEI_LMR;
  const uint32_t slots = lmr ? (uint32_t)(b - 1) : (uint32_t)b;
  const uint32_t top = lmr ? 6u : 7u;

  // ---- my 16 pixels and their labels --------------------------------------------------
  const uint64_t p0 = start + 16u * t;
  int valid = p0 < N ? (int)umin64(16, N - p0) : 0;
  const uint8_t* src = d.src + p0;
  uint32_t px[4] = {0, 0, 0, 0};
  if (valid == 16 && ((reinterpret_cast<uintptr_t>(src) & 15) == 0)) {
    uint4 v = *reinterpret_cast<const uint4*>(src);
    px[0] = v.x; px[1] = v.y; px[2] = v.z; px[3] = v.w;
  } else {
    for (int k = 0; k < valid; k++) px[k >> 2] |= (uint32_t)src[k] << (8 * (k & 3));
  }
  uint32_t zmask;   // bit k set: pixel k is redundant (label 0)
  if (!lmr) {
    zmask = 0;
#pragma unroll
    for (int k = 0; k < 16; k++) zmask |= (((px[k >> 2] >> (8 * (k & 3))) & 1u) ^ 1u) << k;
  } else {
    const uint64_t nw = (N + 31) >> 5;
    const uint32_t lb = stream_bits32(d.map_bits, nw, p0);        // bit k = map bit p0 + k
    zmask = ~lb & 0xFFFFu;
  }
  zmask &= valid >= 16 ? 0xFFFFu : ((1u << valid) - 1u);
  const uint32_t mycnt = (uint32_t)__popc(zmask) * slots;

  // ---- block scan of slot counts ------------------------------------------------------
  uint32_t inc = mycnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t v = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31) warp_tot[warp] = inc;
  if (EXTRACT) for (int i = t; i < EBUF_WORDS; i += HIDE_THREADS) lbuf[i] = 0u;
  __syncthreads();
  uint32_t wbase = 0, T = 0;
#pragma unroll
  for (int i = 0; i < HIDE_THREADS / 32; i++) {
    const uint32_t v = warp_tot[i];
    if (i < warp) wbase += v;
    T += v;
  }
  const uint32_t my_off = wbase + inc - mycnt;       // exclusive, local to the chunk

  // extractor: gather my raw slot bits into the chunk-local stream
  if (EXTRACT) {
    uint32_t o = my_off;
    for (int k = 0; k < 16; k++) {
      if (!((zmask >> k) & 1u)) continue;
      const uint32_t pix = (px[k >> 2] >> (8 * (k & 3))) & 0xFFu;
      const uint32_t field = (pix >> (top + 1 - slots)) & ((1u << slots) - 1u);  // bit `top` first
      or_bits(lbuf, o, field, slots);
      o += slots;
    }
    __syncthreads();
  }

  // ---- publish the aggregate, look back for the offset (warp 0, 32 chunks a step) ----
  if (warp == 0) {
    uint32_t tail = 0;
    if (EXTRACT && T > 0) tail = T >= 32 ? get_bits(lbuf, T - 32, 32) : get_bits(lbuf, 0, T);
    unsigned long long* st = B.chunk_status + g;
    uint32_t G = 0, acc = 0;
    if (c == 0) {
      if (lane == 0) st_release_u64(st, pack_status(2, T, tail));
    } else {
      if (lane == 0) st_release_u64(st, pack_status(1, T, tail));
      uint32_t have = 0;
      int64_t cur = (int64_t)g - 1;                  // predecessor seen by lane 0
      const int64_t first = (int64_t)d.chunk_base;   // the image's chunk 0 is always inclusive
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
        const int L = incm ? __ffs(incm) - 1 : 31;     // lanes 0..L lie after the nearest inclusive one
        const uint32_t v = lane <= L ? ((uint32_t)(sw >> 32) & 0x3FFFFFFFu) : 0u;
        const uint32_t tl = (uint32_t)sw;
        uint32_t sum = v;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        G += sum;
        // the last 32 raw bits before this chunk: nearest predecessors first
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
        if (incm) break;
        cur -= 32;
      }
      uint32_t itail = acc;                          // last 32 raw bits before G + T
      if (EXTRACT) {
        if (T >= 32) itail = tail;
        else if (T > 0) itail = (acc << T) | tail;
      }
      if (lane == 0) st_release_u64(st, pack_status(2, G + T, itail));
    }
    if (lane == 0) { s_G = G; s_carry = acc; s_T = T; }
  }
  __syncthreads();
  const uint64_t G = s_G;
  const uint64_t Gend = G + T;
  const bool last = c + 1 == d.nchunks;
  if (last && t == 0) {
    if (EXTRACT) info->extracted = umin64(d.max_bits, Gend);
    else {
      info->embedded = umin64(d.nbits, Gend);
      if (d.nbits > Gend) { info->status = ERR_CAPACITY; set_error(B.err, ERR_CAPACITY); }
    }
  }

  // ---- keystream words z2 covering the words this chunk touches ----------------------
  // embed: payload bits [G, min(Gend, nbits)); extract: output words of this chunk
  uint64_t w_lo, w_hi;   // inclusive word range (w_hi < w_lo: none)
  if (EXTRACT) {
    // words whose last bit lies in [G, Gend); the image's last chunk also writes the
    // final partial word; only words that start below max_bits
    w_lo = G >> 5;
    uint64_t hi_excl = Gend >> 5;
    if (last && (Gend & 31)) hi_excl += 1;
    const uint64_t lim = (d.max_bits + 31) >> 5;
    if (hi_excl > lim) hi_excl = lim;
    if (hi_excl > w_lo) w_hi = hi_excl - 1;
    else { w_lo = 1; w_hi = 0; }
  } else {
    const uint64_t end = umin64(Gend, d.nbits);
    if (end > G) { w_lo = G >> 5; w_hi = (end - 1) >> 5; }
    else { w_lo = 1; w_hi = 0; }
  }
  const bool any = w_hi >= w_lo;
  const uint64_t blk0 = any ? (w_lo >> 4) : 0;
  const uint32_t nblk = any ? (uint32_t)((w_hi >> 4) - blk0 + 1) : 0u;
  // spread the ChaCha blocks over the warps
  for (uint32_t j = t; j < nblk; j += HIDE_THREADS) {
    {                        // consecutive lanes: few, full warps
      uint32_t o[16];
      chacha20_block(d.k2, (uint32_t)(blk0 + j), d.n2, o);
#pragma unroll
      for (int k = 0; k < 16; k++) ebuf[16 * j + k] = bswap32(o[k]);
    }
  }
  __syncthreads();
  const uint64_t wb = blk0 * 16;                   // global word of ebuf[0]

  if (!EXTRACT) {
    // encrypted payload e = m XOR z2 (Sec. III-A-2: the hider encrypts with K2)
    if (any) {
      const uint64_t pw = (d.nbits + 31) >> 5;
      const uint32_t* pay = reinterpret_cast<const uint32_t*>(d.payload);
      for (uint64_t w = w_lo + t; w <= w_hi; w += HIDE_THREADS)
        if (w < pw) ebuf[w - wb] ^= bswap32(__ldg(pay + w));
    }
    if (t == 0) ebuf[nblk * 16] = 0u;
    __syncthreads();
    uint64_t k = G + my_off;
    for (int q = 0; q < 16; q++) {
      if (!((zmask >> q) & 1u)) continue;
      if (k >= d.nbits) break;
      const uint32_t n = (uint32_t)umin64(slots, d.nbits - k);
      const uint32_t e = get_bits(ebuf, (uint32_t)(k - 32 * wb), n);
      const uint32_t sh = top + 1 - n;                   // first bit into bit `top`
      const uint32_t m = ((1u << n) - 1u) << sh;
      uint32_t& w = px[q >> 2];
      const uint32_t bs = 8 * (q & 3);
      w = (w & ~(m << bs)) | ((e << sh) << bs);
      k += slots;
    }
    uint8_t* dst = d.dst + p0;
    if (valid == 16 && ((reinterpret_cast<uintptr_t>(dst) & 15) == 0)) {
      *reinterpret_cast<uint4*>(dst) = make_uint4(px[0], px[1], px[2], px[3]);
    } else {
      for (int k2 = 0; k2 < valid; k2++) dst[k2] = (uint8_t)(px[k2 >> 2] >> (8 * (k2 & 3)));
    }
  } else {
    // output words: raw stream bits (earlier chunks' tail + mine), XOR z2, masked to
    // min(max_bits, Gend) bits
    const uint64_t limit = umin64(d.max_bits, Gend);
    uint32_t* out = reinterpret_cast<uint32_t*>(d.bits_out);
    const uint32_t carry = s_carry;
    for (uint64_t w = w_lo + t; any && w <= w_hi; w += HIDE_THREADS) {
      const uint64_t b0 = 32 * w;
      uint32_t raw;
      if (b0 >= G) {
        raw = get_bits(lbuf, (uint32_t)(b0 - G), 32);
      } else {
        const uint32_t k = (uint32_t)(G - b0);             // 1..31 bits from earlier chunks
        raw = ((carry & ((1u << k) - 1u)) << (32 - k)) | (lbuf[0] >> k);
      }
      uint32_t val = raw ^ ebuf[w - wb];
      if (b0 + 32 > limit) {
        const uint64_t keep = limit > b0 ? limit - b0 : 0;
        val = keep == 0 ? 0u : (val & (0xFFFFFFFFu << (32 - keep)));
      }
      out[w] = bswap32(val);
    }
  }
}

// LMR side information into bit 7 (Sec. III-B-1): pixel q < side_nbits.
__global__ void k_lmr_side(Batch B) {
  const uint32_t g = blockIdx.x;
  const int img = owner_of(B.chunk_prefix, B.n_images, g);
  const ImgDesc& d = B.desc[img];
  const uint64_t N = (uint64_t)d.H * d.W;
  const uint64_t p0 = (uint64_t)(g - d.chunk_base) * CHUNK_PX + 16u * threadIdx.x;
  if (p0 >= N || p0 >= d.side_nbits || !d.side_bits) return;
  const int n = (int)umin64(umin64(16, N - p0), d.side_nbits - p0);
  const uint32_t sb = stream_bits32(d.side_bits, (d.side_nbits + 31) >> 5, p0);
  for (int k = 0; k < n; k++) d.dst[p0 + k] = (uint8_t)((d.dst[p0 + k] & 0x7Fu) | (((sb >> k) & 1u) << 7));
}

void launch_hide(const Batch& B, bool extract, cudaStream_t st) {
  if (B.total_chunks == 0) return;
  if (extract) k_hide<true><<<B.total_chunks, HIDE_THREADS, 0, st>>>(B);
  else k_hide<false><<<B.total_chunks, HIDE_THREADS, 0, st>>>(B);
}
void launch_lmr_side(const Batch& B, cudaStream_t st) {
  if (B.total_chunks == 0) return;
  k_lmr_side<<<B.total_chunks, HIDE_THREADS, 0, st>>>(B);
}

}  // namespace rdhei
