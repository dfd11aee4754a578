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
#include "slots.cuh"

namespace rdhei {

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
  __shared__ SlotTables tabs;
  const int t = threadIdx.x;
  init_slot_tables(tabs);
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
      spread_slots(cur.px, zmask, slots, fshift, sbuf, 32 * w_lo, G + my_off, d.nbits, tabs, B.err);
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
      gather_slots(cur.px, zmask, slots, fshift, my_off, sbuf, tabs, B.err);
      __syncthreads();
      // words of [G, min(G + T, E)), E = bits the receiver asked for and the image holds
      const uint64_t E = info->extracted;
      const uint64_t end = umin64(G + T, E);
      uint32_t* out = reinterpret_cast<uint32_t*>(d.bits_out);
      if (end > G) {
        // in 32-bit offsets from word w_lo, as in the fused extraction: word w_lo + k is
        // sbuf's words k - 1, k shifted right by G's offset inside word w_lo
        const uint32_t nwords = (uint32_t)(((end - 1) >> 5) - w_lo) + 1;
        const uint32_t g0 = (uint32_t)(G & 31), e = (uint32_t)(end - 32 * w_lo);
        uint32_t* const outw = out + w_lo;
        for (uint32_t k = t; k < nwords; k += HIDE_THREADS) {
          const uint32_t b0 = 32 * k;
          const uint32_t lo = b0 > g0 ? b0 : g0, hi = b0 + 32 < e ? b0 + 32 : e;   // my bits of word w_lo + k
          if (!RDHEI_IDX_OK(B.err, w_lo + k < ((d.max_bits + 31) >> 5) && k < SBUF_WORDS)) continue;
          const uint32_t x = __funnelshift_r(sbuf[k], k > 0 ? sbuf[k - 1] : 0u, g0);
          const uint32_t keep = (0xFFFFFFFFu >> (lo - b0)) & ~(hi - b0 >= 32 ? 0u : 0xFFFFFFFFu >> (hi - b0));
          if (lo == b0 && hi == b0 + 32) outw[k] = bswap32(x);
          else atomicOr(outw + k, bswap32(x & keep));
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

// Fused decode, K2 half (Sec. III-A-3 / III-B-3, "receiver has only K2", run inside
// the both-keys decode): one CTA per part of a 64-row strip of the marked image (rows
// B.part_rows at a time; a whole strip by default).  Each part's slots start at the
// stream bit k_topmap derived from label counts of the first pass (per tile, or per
// tile row for split strips), so the CTA walks its 8192-pixel chunks in raster order
// with a running offset -- no count pass, no cross-CTA wait.  The K2 keystream is
// staged in a window of up to 256 ChaCha20 blocks, one block per thread: the first
// window while the first chunk's loads are in flight, the next one whenever a chunk's
// output words run past it (wide strips).  Each chunk's slots are gathered into shared
// memory, XOR-ed with the keystream and stored: words inside the chunk's range whole,
// words shared with a neighbouring chunk or CTA with atomicOr into words that start at
// zero (cleared by k_topmap at part and strip ends, here at chunk ends).
constexpr int Z2_WINDOW_BLOCKS = HIDE_THREADS;   // 256 keystream blocks = 4096 words
static_assert(16 * Z2_WINDOW_BLOCKS >= Z2BUF_WORDS, "a window holds one chunk's keystream");

// keystream words of blocks [j0, j0 + nblk) into z2 (one block per thread)
// Block t goes to words 16 t .. 16 t + 15 as four 16-byte stores, its 16-byte chunk q at
// chunk q ^ ((t >> 1) & 3): the eight threads of a store phase then hit distinct banks
// (plain layout: 16 threads per bank pair).  Word w of the window is read at z2_word(w).
__device__ __forceinline__ uint32_t z2_word(uint32_t w) { return w ^ ((w >> 3) & 0xCu); }
__device__ __forceinline__ void z2_blocks(const ImgDesc& d, uint64_t j0, uint32_t nblk, uint32_t* z2) {
  const int t = threadIdx.x;
  if ((uint32_t)t < nblk) {
    uint32_t o[16];
    chacha20_block<2>(d.k2, (uint32_t)(j0 + t), d.n2, o, d.one);
    uint4* b = reinterpret_cast<uint4*>(z2 + 16 * t);
    const int sw = (t >> 1) & 3;
#pragma unroll
    for (int q = 0; q < 4; q++) b[q ^ sw] = make_uint4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
  }
}

// blocks of the window that starts at block j0: up to Z2_WINDOW_BLOCKS, not past the
// block of the strip's last slot
__device__ __forceinline__ uint32_t z2_window(uint64_t j0, uint64_t send) {
  return (uint32_t)umin64(Z2_WINDOW_BLOCKS, (((send - 1) >> 5) >> 4) - j0 + 1);
}

// Five CTAs per SM (48 registers) with each chunk's loads at the top of its iteration
// measured faster than four (64 registers) with the next chunk's loads in flight during
// the current one: 0.231 -> 0.219 ms on 1000 x 512^2.
__global__ void __launch_bounds__(HIDE_THREADS, 5) k_extract_strips(Batch B) {
  pdl_wait();      // the previous kernel of the operation has finished
  pdl_trigger();
  __shared__ uint32_t sbuf[SBUF_WORDS];
  __shared__ __align__(16) uint32_t z2buf[16 * Z2_WINDOW_BLOCKS];
  __shared__ uint32_t warp_tot[HIDE_THREADS / 32];
  __shared__ SlotTables tabs;
  const int t = threadIdx.x;
  init_slot_tables(tabs);
  const uint32_t R = (uint32_t)B.part_rows, parts = TILE / R;
  const uint32_t s = blockIdx.x / parts, part = blockIdx.x % parts;
  const int img = (int)__ldg(B.strip_owner + s);
  const ImgDesc& d = B.desc[img];
  const rdhei_info* info = reinterpret_cast<const rdhei_info*>(d.info);
  const uint32_t ty = s - __ldg(B.strip_prefix + img);
  const uint64_t W = (uint64_t)d.W;
  const uint32_t rows = (uint32_t)min(TILE, d.H - (int)ty * TILE);
  const uint32_t r0 = part * R, r1 = min(r0 + R, rows);
  if (r0 >= rows) return;                                    // uniform: the strip has no such rows
  const uint32_t slots = (uint32_t)slots_of(d, info);
  uint64_t G0 = B.strip_base[s], Gend = G0 + B.strip_tot[s];
  if (parts > 1) {
    const uint32_t* pb = B.part_base + (size_t)s * MAX_PARTS;
    G0 = pb[part];
    if (r1 < rows) Gend = pb[part + 1];                      // else the strip's end
  }
  const uint64_t p0 = ((uint64_t)ty * TILE + r0) * W, p1 = ((uint64_t)ty * TILE + r1) * W;
  const uint64_t send = umin64(Gend, info->extracted);
  if (G0 >= send) return;                                    // uniform: no slots to read
  const uint32_t fshift = (d.variant == RDHEI_LMR ? 7u : 8u) - slots;
  uint32_t* out = reinterpret_cast<uint32_t*>(d.bits_out);
  const uint64_t out_words = (d.max_bits + 31) >> 5;
  (void)out_words;                                           // index checks only
  // 32-bit positions: pixels from the part's first (p0), stream bits from 32 W0, the
  // start of the word holding its first slot bit; K2 blocks from J0 = W0 / 16
  const uint64_t W0 = G0 >> 5, J0 = W0 >> 4;
  const uint32_t o0 = (uint32_t)(W0 & 15);                    // W0's word inside block J0
  const uint8_t* const ssrc = d.src + p0;
  const uint32_t npx = (uint32_t)(p1 - p0), send_r = (uint32_t)(send - 32 * W0);
  uint32_t* const outp = out + W0;
  // the part's first keystream window
  uint32_t jb = 0;                                           // window: blocks [J0 + jb, J0 + jb + Jn)
  uint32_t Jn = z2_window(J0, send);
  z2_blocks(d, J0, Jn, z2buf);
  __syncthreads();   // tables, keystream
  uint32_t g = (uint32_t)(G0 & 31);
  for (uint32_t c0 = 0; c0 < npx && g < send_r; c0 += SCAN_PX) {
    ChunkPx cur;
    load_strip_run<false>(d, ssrc, p0, c0 + (uint32_t)HIDE_PX * t, npx, cur);
    const uint32_t zmask = zero_mask(d, cur);
    uint32_t Tc;
    const uint32_t my_off = block_exclusive_scan((uint32_t)__popc(zmask) * slots, warp_tot, Tc);
    const uint32_t endc = min(g + Tc, send_r);
    if (endc > g) {
      for (int i = t; i < (int)((Tc >> 5) + 2) && i < SBUF_WORDS; i += HIDE_THREADS) sbuf[i] = 0u;
      const uint32_t wa = g >> 5, wb = (endc - 1) >> 5;       // words, from W0
      if (((o0 + wb) >> 4) >= jb + Jn) {
        // the chunk's words run past the window: the next window starts at its first block
        // (the block scan's barriers ordered every earlier read of z2buf)
        jb = (o0 + wa) >> 4;
        Jn = z2_window(J0 + jb, send);
        z2_blocks(d, J0 + jb, Jn, z2buf);
      }
      // a word that starts inside this chunk and ends inside the next one of this part
      // is cleared here, before the ORs of both; the word holding the part's end (shared
      // with the next part or strip, or the last one) was cleared by k_topmap
      if (t == 0 && (endc & 31) && ((endc >> 5) << 5) >= g && (endc >> 5) < (send_r >> 5) &&
          RDHEI_IDX_OK(B.err, W0 + (endc >> 5) < out_words))
        outp[endc >> 5] = 0u;
      __syncthreads();
      gather_slots(cur.px, zmask, slots, fshift, my_off, sbuf, tabs, B.err);
      __syncthreads();
      // output words wa .. wb: the chunk's stream starts g0 bits into word wa, so word
      // wa + k is sbuf's words k - 1, k shifted right by g0 (bits outside [g, endc)
      // masked off)
      const uint32_t nwords = wb - wa + 1;
      const uint32_t g0 = g & 31, e = endc - 32 * wa;
      const uint32_t zoff = o0 + wa - 16 * jb;                  // z2buf word of output word wa
      uint32_t* const outw = outp + wa;
      for (uint32_t k = t; k < nwords; k += HIDE_THREADS) {
        const uint32_t b0 = 32 * k;
        const uint32_t lo = b0 > g0 ? b0 : g0, hi = b0 + 32 < e ? b0 + 32 : e;   // my bits of word wa + k
        if (!RDHEI_IDX_OK(B.err, W0 + wa + k < out_words && k < SBUF_WORDS &&
                                     zoff + k < (uint32_t)(16 * Z2_WINDOW_BLOCKS)))
          continue;
        const uint32_t x = __funnelshift_r(sbuf[k], k > 0 ? sbuf[k - 1] : 0u, g0);
        const uint32_t keep = (0xFFFFFFFFu >> (lo - b0)) & ~(hi - b0 >= 32 ? 0u : 0xFFFFFFFFu >> (hi - b0));
        const uint32_t v = bswap32(x & keep) ^ (z2buf[z2_word(zoff + k)] & bswap32(keep));
        if (lo == b0 && hi == b0 + 32) outw[k] = v;
        else atomicOr(outw + k, v);
      }
    }
    g += Tc;
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
  const uint32_t sb = stream_bits32(d.side_bits, (uint32_t)((d.side_nbits + 31) >> 5), (uint32_t)p0);
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
void launch_extract_strips(const Batch& B, cudaStream_t st) {
  if (B.total_strips == 0) return;
  launch_pdl(k_extract_strips, dim3(B.total_strips * (TILE / B.part_rows)), dim3(HIDE_THREADS), 0, st, B);
}
void launch_lmr_side(const Batch& B, cudaStream_t st) {
  if (B.total_chunks == 0) return;
  launch_pdl(k_lmr_side, dim3(B.total_chunks), dim3(HIDE_THREADS), 0, st, B);
}

}  // namespace rdhei
