// pass1.cu -- first pass over every 64 x 64 tile: keystream, rotation angles of the
// levels inside the tile, label histogram (owner) or decryption (K1 receiver).
//
// One thread owns one 64-pixel tile row: it computes the ChaCha20 block(s) covering
// that row of the keystream s (Sec. "Secret key generation"), so every keystream byte
// of the image is computed exactly once per call.  Block sums of s give the
// quarter-turn angles of Eq. (roration) for levels 1..6 (blocks inside the tile);
// the tile total feeds the levels above (topmap.cu).
//
//   owner (MODE_ENC):  stash := s; label histogram of Eqs. (gliding1/2) from I.
//   K1 receiver (MODE_DEC): stash := I_e' XOR s with the location map bit kept
//        (EMR: LSB = map, aux plane = LSB of s; LMR: bit 7 = map l, aux = eta).
#include "common.cuh"

namespace rdhei {

enum { MODE_ENC = 0, MODE_DEC = 1 };

// mod-4 addition of 32 packed 2-bit lanes: per lane the low bit is a0 ^ b0 and the
// high bit a1 ^ b1 ^ (a0 & b0); the carries (a & b & low-bit mask) << 1 land on high
// bits only, so one three-way XOR combines them
__device__ __forceinline__ uint64_t add4(uint64_t a, uint64_t b) {
  const uint64_t L = 0x5555555555555555ull;
  return a ^ b ^ ((a & b & L) << 1);
}
// 4-bit field at bits 28..31 of x shifted into the bottom of acc (acc << 4 | x >> 28)
__device__ __forceinline__ uint32_t push_nibble(uint32_t acc, uint32_t x) { return __funnelshift_l(x, acc, 4); }
// pairwise (mod 4) sums of adjacent 2-bit lanes, compacted: 2k lanes -> k lanes
__device__ __forceinline__ uint64_t pair4(uint64_t v) {
  const uint64_t M = 0x3333333333333333ull;
  uint64_t s = ((v & M) + ((v >> 2) & M)) & M;        // lane k in nibble k (2 bits used)
  s = (s | (s >> 2)) & 0x0F0F0F0F0F0F0F0Full;
  s = (s | (s >> 4)) & 0x00FF00FF00FF00FFull;
  s = (s | (s >> 8)) & 0x0000FFFF0000FFFFull;
  s = (s | (s >> 16)) & 0x00000000FFFFFFFFull;
  return s;
}
// The same on 32-bit words: from level 2 on a 64-pixel row has at most 16 lanes.
__device__ __forceinline__ uint32_t add4_32(uint32_t a, uint32_t b) { return a ^ b ^ ((a & b & 0x55555555u) << 1); }
__device__ __forceinline__ uint32_t pair4_32(uint32_t v) {
  const uint32_t M = 0x33333333u;
  uint32_t s = ((v & M) + ((v >> 2) & M)) & M;
  s = (s | (s >> 2)) & 0x0F0F0F0Fu;
  s = (s | (s >> 4)) & 0x00FF00FFu;
  s = (s | (s >> 8)) & 0x0000FFFFu;
  return s;
}
__device__ __forceinline__ uint64_t shfl_xor64(uint64_t v, int m) {
  uint32_t lo = __shfl_xor_sync(0xffffffffu, (uint32_t)v, m);
  uint32_t hi = __shfl_xor_sync(0xffffffffu, (uint32_t)(v >> 32), m);
  return ((uint64_t)hi << 32) | lo;
}

// 20 CTAs per SM (48 registers) measured slightly faster than the unbounded build
// (56-63 registers) and than 12
template <int N>
struct LevelTag {
  static constexpr int value = N;
};

// Row partial sums at level SH + 2 (2^SH keystream words per 2-bit lane), the shift a
// compile-time constant so that the loop's lane tests and shifts fold away.
template <int SH>
__device__ __forceinline__ uint64_t level_partial(const uint32_t (&sw)[16]) {
  uint64_t v = 0;
  uint32_t acc = 0;
#pragma unroll
  for (int i = 0; i < 16; i++) {
    acc += sw[i] & 0x03030303u;                            // byte lanes, <= 12 each
    if (((i + 1) & ((1 << SH) - 1)) == 0) {
      const uint32_t lanev = ((acc * 0x01010101u) >> 24) & 3u;   // sum of the 4 bytes, mod 4
      v |= (uint64_t)lanev << (2 * (i >> SH));
      acc = 0;
    }
  }
  return v;
}

template <int MODE, bool GENERAL, bool ANY_MED>
__global__ void __launch_bounds__(64, 20) k_pass1(Batch B) {
  pdl_wait();      // the previous kernel of the operation has finished
  pdl_trigger();
  // keystream staging for rows that straddle two ChaCha blocks (W not a multiple of 64)
  __shared__ uint32_t ks_stage[GENERAL ? 64 : 1][33];
  __shared__ __align__(16) uint8_t sub[SUBTREE_BYTES];
  __shared__ uint64_t l6_part[2];
  __shared__ uint32_t zero_cnt[2][8];

  const uint32_t g = blockIdx.x;
  const int img = (int)__ldg(B.tile_owner + g);
  const ImgDesc& d = B.desc[img];
  const uint32_t t_local = g - d.tile_base;
  const int ty = (int)(t_local / d.tiles_x), tx = (int)(t_local % d.tiles_x);
  const int r = threadIdx.x, lane = r & 31, warp = r >> 5;
  const int H = d.H, W = d.W;
  const int y = ty * TILE + r, x0 = tx * TILE;
  const bool row_ok = y < H;
  const int len = row_ok ? min(TILE, W - x0) : 0;
  const uint32_t base = (uint32_t)y * (uint32_t)W + (uint32_t)x0;   // < 2^28: 32-bit positions

  for (int i = r; i < SUBTREE_BYTES / 4; i += 64) reinterpret_cast<uint32_t*>(sub)[i] = 0u;

  // ---- keystream of this tile row -------------------------------------------------
  uint32_t sw[16];
  const bool aligned = ((base & 63) == 0) && len == TILE;
  if (len == 0) {
#pragma unroll
    for (int i = 0; i < 16; i++) sw[i] = 0u;
  } else if (aligned || !GENERAL) {
    chacha20_block<2>(d.k1, base >> 6, d.n1, sw, d.one);
  } else {
    // the row straddles two ChaCha blocks: stage both and pick the 64 bytes
    uint32_t o[16];
    const uint32_t b0 = base >> 6;
    const int off = (int)(base & 63);
    if (len > 0) {
      chacha20_block<2>(d.k1, (uint32_t)b0, d.n1, o, d.one);
#pragma unroll
      for (int i = 0; i < 16; i++) ks_stage[r][i] = o[i];
      if (off + len > 64) {
        chacha20_block<2>(d.k1, (uint32_t)(b0 + 1), d.n1, o, d.one);
#pragma unroll
        for (int i = 0; i < 16; i++) ks_stage[r][16 + i] = o[i];
      } else {
#pragma unroll
        for (int i = 0; i < 16; i++) ks_stage[r][16 + i] = 0u;
      }
      ks_stage[r][32] = 0u;
    }
    const int wsh = off >> 2, bsh = (off & 3) * 8;
#pragma unroll
    for (int i = 0; i < 16; i++) {
      uint32_t v = 0;
      if (len > 0) {
        uint32_t lo = ks_stage[r][wsh + i], hi = ks_stage[r][wsh + i + 1];
        v = bsh ? __funnelshift_r(lo, hi, bsh) : lo;
      }
      // clear bytes past the row end
      int valid = len - 4 * i;
      if (valid <= 0) v = 0;
      else if (valid < 4) v &= (1u << (8 * valid)) - 1u;
      sw[i] = v;
    }
  }

  // ---- row data: owner reads I (histogram), receiver reads I_e' -------------------
  uint32_t px[16];
  const uint8_t* src = d.src + base;
  const bool vec = aligned && ((reinterpret_cast<uintptr_t>(src) & 15) == 0);
  if (vec) {
    const uint4* s4 = reinterpret_cast<const uint4*>(src);
#pragma unroll
    for (int q = 0; q < 4; q++) {
      uint4 v = __ldg(s4 + q);
      px[4 * q] = v.x; px[4 * q + 1] = v.y; px[4 * q + 2] = v.z; px[4 * q + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < 16; i++) {
      uint32_t v = 0;
#pragma unroll
      for (int k = 0; k < 4; k++) {
        int c = 4 * i + k;
        if (c < len) v |= (uint32_t)__ldg(src + c) << (8 * k);
      }
      px[i] = v;
    }
  }

  if (MODE == MODE_ENC) {
    // stash the keystream for the gather pass
    uint8_t* st = d.stash + base;
    if (len > 0) {
      if (vec && ((reinterpret_cast<uintptr_t>(st) & 15) == 0)) {
        uint4* s4 = reinterpret_cast<uint4*>(st);
#pragma unroll
        for (int q = 0; q < 4; q++) s4[q] = make_uint4(sw[4 * q], sw[4 * q + 1], sw[4 * q + 2], sw[4 * q + 3]);
      } else {
#pragma unroll
        for (int c = 0; c < 64; c++)
          if (c < len) st[c] = (uint8_t)(sw[c >> 2] >> (8 * (c & 3)));
      }
    }
    // label histogram: zeros(b) = #pixels whose top b bits equal the left neighbour's
    // (Eqs. gliding1/2 with the left-neighbour form of the map).  The first image
    // column has no left neighbour and is never redundant.  MED variant (related
    // work): the prediction is the median edge detector of the left, upper and
    // upper-left pixels instead (row 0: left; column 0: upper; pixel (0, 0): none).
    uint32_t left;
    if (len > 0) left = x0 > 0 ? (uint32_t)__ldg(src - 1) : ((px[0] & 0xFFu) ^ 0xFFu);
    else left = 0;
    const bool med = ANY_MED && d.med != 0 && len > 0;
    const bool seven = d.variant == 0;                     // EMR predicts on the top seven bits
    uint32_t up[16], ul = 0;
    if (med) {
      if (y > 0) {
        const uint8_t* us = src - W;
        if (vec && ((reinterpret_cast<uintptr_t>(us) & 15) == 0)) {
          const uint4* u4 = reinterpret_cast<const uint4*>(us);
#pragma unroll
          for (int q = 0; q < 4; q++) {
            const uint4 v = __ldg(u4 + q);
            up[4 * q] = v.x; up[4 * q + 1] = v.y; up[4 * q + 2] = v.z; up[4 * q + 3] = v.w;
          }
        } else {
#pragma unroll
          for (int i = 0; i < 16; i++) {
            uint32_t v = 0;
#pragma unroll
            for (int k = 0; k < 4; k++)
              if (4 * i + k < len) v |= (uint32_t)__ldg(us + 4 * i + k) << (8 * k);
            up[i] = v;
          }
        }
        ul = x0 > 0 ? (uint32_t)__ldg(us - 1) : 0u;
      } else {
#pragma unroll
        for (int i = 0; i < 16; i++) up[i] = 0u;
      }
      if (x0 == 0) left = 0;
    }
    uint32_t nz[8];
#pragma unroll
    for (int k = 0; k < 8; k++) nz[k] = 0;
#pragma unroll
    for (int i = 0; i < 16; i++) {
      uint32_t prev = i == 0 ? (left << 24) : px[i - 1];
      uint32_t pred = __funnelshift_l(prev, px[i], 8);          // left neighbours
      if (med) {
        const uint32_t Bw = up[i], C = __funnelshift_l(i == 0 ? (ul << 24) : up[i - 1], up[i], 8);
        // EMR: the median of the values with the LSB cleared (twice that of the top seven bits)
        const uint32_t keep = seven ? 0xFEFEFEFEu : 0xFFFFFFFFu;
        uint32_t m = med4(pred & keep, Bw & keep, C & keep);
        if (y == 0) m = seven ? pred & 0xFEFEFEFEu : pred;      // row 0: from the left
        if (i == 0 && x0 == 0) m = (m & 0xFFFFFF00u) | (Bw & (seven ? 0xFEu : 0xFFu));   // column 0: from above
        pred = m;
      }
      uint32_t dd = px[i] ^ pred;
      if (med && i == 0 && x0 == 0 && y == 0) dd |= 0xFFu;       // pixel (0, 0): never redundant
      if (GENERAL) {
        // bytes past the row end count as "differs"; without GENERAL every row is 64
        // pixels long or empty, and an empty row is zeroed below
        const int valid = len - 4 * i;
        if (valid < 4) dd |= valid <= 0 ? 0xFFFFFFFFu : (0xFFFFFFFFu << (8 * valid));
      }
      // nz[b - 1] += 128 per pixel whose top b bits differ (the flag byte 0x80 summed by
      // a byte dot product with 1, 1, 1, 1)
      uint32_t m = dd & 0x7F7F7F7Fu;
      nz[0] = __dp4a(dd & 0x80808080u, 0x01010101u, nz[0]);               // b = 1
#pragma unroll
      for (int b = 2; b <= 8; b++) {
        const uint32_t K = (0x80u - (0x100u >> b)) * 0x01010101u;            // top b bits nonzero
        nz[b - 1] = __dp4a(((m + K) | dd) & 0x80808080u, 0x01010101u, nz[b - 1]);
      }
    }
    // per-row zero counts = valid pixels - nonzero ones; reduce over the CTA
#pragma unroll
    for (int k = 0; k < 8; k += 2) {
      // the 64 examined bytes include the padding past the row end, all "differs";
      // two counts (<= 64 a row, <= 2048 a warp) in the halves of one word
      const uint32_t z0 = (GENERAL || len > 0) ? 64u - (nz[k] >> 7) : 0u;
      const uint32_t z1 = (GENERAL || len > 0) ? 64u - (nz[k + 1] >> 7) : 0u;
      const uint32_t z = __reduce_add_sync(0xffffffffu, z0 | (z1 << 16));
      if (lane == 0) { zero_cnt[warp][k] = z & 0xFFFFu; zero_cnt[warp][k + 1] = z >> 16; }
    }
  } else {
    // K1 receiver: decrypt into the stash, keep the map bit, and record the aux plane.
    // Also counts this row's label-0 pixels, the payload slots a K2 receiver reads (EMR:
    // LSB 0; LMR: map bit 0); the fused decode sums them per strip.
    uint64_t auxbits = 0;
    uint32_t zrow = 0;
    uint8_t* st = d.stash + base;
    if (d.variant == 0) {
      // the LSBs of s, pixel 4i+k -> aux bit 4i+k: the multiply gathers a word's four
      // LSBs into bits 28..31 (bit 8k -> 28+k, no overlapping partial products), and the
      // words are shifted in from the last one down
      uint32_t alo = 0, ahi = 0;
#pragma unroll
      for (int i = 15; i >= 0; i--) {
        const uint32_t s = sw[i];
        zrow = __dp4a(~px[i] & 0x01010101u, 0x01010101u, zrow);   // slot pixels: LSB 0 (FMA pipe)
        px[i] ^= s & 0xFEFEFEFEu;                       // bits 7..1 decrypted, LSB = map l
        const uint32_t x = (s & 0x01010101u) * 0x10204080u;
        if (i >= 8) ahi = push_nibble(ahi, x);
        else alo = push_nibble(alo, x);
      }
      auxbits = ((uint64_t)ahi << 32) | alo;
      zrow -= (uint32_t)(64 - len);                     // bytes past the row end were loaded as 0
    } else {
      const uint32_t nw = ((uint32_t)H * (uint32_t)W + 31) >> 5, pb = base;
      uint32_t lb0 = len > 0 ? stream_bits32(d.map_bits, nw, pb) : 0u;
      uint32_t lb1 = len > 32 ? stream_bits32(d.map_bits, nw, pb + 32) : 0u;
      uint32_t eb0 = len > 0 ? stream_bits32(d.eta_bits, nw, pb) : 0u;
      uint32_t eb1 = len > 32 ? stream_bits32(d.eta_bits, nw, pb + 32) : 0u;
      uint64_t lb = ((uint64_t)lb1 << 32) | lb0, eb = ((uint64_t)eb1 << 32) | eb0;
#pragma unroll
      for (int i = 0; i < 16; i++) {
        uint32_t nib = (uint32_t)(lb >> (4 * i)) & 0xFu;
        uint32_t lbytes = ((nib * 0x00204081u) & 0x01010101u) << 7;
        px[i] = ((px[i] ^ sw[i]) & 0x7F7F7F7Fu) | lbytes;   // bits 6..0 decrypted, bit 7 = map l
      }
      auxbits = eb;
      const uint64_t valid = len >= 64 ? ~0ull : ((1ull << len) - 1ull);
      zrow = (uint32_t)__popcll(~lb & valid);
    }
    // per tile row, for the fused decode's split strips (written whatever the split, so
    // that a plan may change its split between runs of the later stages)
    if (B.count_rows) B.rowcnt[(size_t)g * TILE + r] = (uint8_t)zrow;
    zrow = __reduce_add_sync(0xffffffffu, zrow);
    if (lane == 0) zero_cnt[warp][0] = zrow;
    if (len < 64) auxbits &= len > 0 ? ((len == 64) ? ~0ull : ((1ull << len) - 1)) : 0ull;
    if (len > 0) {
      if (vec && ((reinterpret_cast<uintptr_t>(st) & 15) == 0)) {
        uint4* s4 = reinterpret_cast<uint4*>(st);
#pragma unroll
        for (int q = 0; q < 4; q++) s4[q] = make_uint4(px[4 * q], px[4 * q + 1], px[4 * q + 2], px[4 * q + 3]);
      } else {
#pragma unroll
        for (int c = 0; c < 64; c++)
          if (c < len) st[c] = (uint8_t)(px[c >> 2] >> (8 * (c & 3)));
      }
    }
    reinterpret_cast<uint64_t*>(B.aux + (size_t)g * AUX_BYTES)[r] = auxbits;
  }

  // ---- block sums of s at levels 1..6 -------------------------------------------------
  // Levels below lmin are never rotated, so the sums start at level Ls = min(max(lmin,1), 4)
  // (LMR's default lmin is 4).  Row partial at level Ls: lane k (2 bits, bits 2k..2k+1) =
  // sum over the row's columns [k 2^Ls, (k+1) 2^Ls) of s mod 4.
  const int lmin = d.lmin;
  // the starting level as a compile-time constant: the partial sums, the row shuffles
  // and the level loop's tests fold for each of the four starting levels
  auto levels = [&](auto ls_tag) {
    constexpr int Ls = decltype(ls_tag)::value;
    uint64_t v = 0;
    if constexpr (Ls == 1) {
      // per word: (t * 0x101) has c0+c1 in byte 1 and c2+c3 in byte 3 (each <= 6, no
      // carries between bytes); their low two bits move to bits 28..29 and 30..31 with
      // one more multiply (bits 8 -> 28 by 2^20, bits 24 -> 30 by 2^6), then shift in
      uint32_t vlo = 0, vhi = 0;
#pragma unroll
      for (int i = 15; i >= 0; i--) {
        const uint32_t u = (sw[i] & 0x03030303u) * 0x0101u;
        const uint32_t x = (u & 0x03000300u) * 0x00100040u;
        if (i >= 8) vhi = push_nibble(vhi, x);
        else vlo = push_nibble(vlo, x);
      }
      v = ((uint64_t)vhi << 32) | vlo;
    } else {
      v = level_partial<Ls - 2>(sw);
    }
    // rows below level Ls; from level 2 on the lanes fit in 32 bits
    uint32_t v32 = 0;
    if constexpr (Ls == 1) {
      v = add4(v, shfl_xor64(v, 1));                       // level 1: 32 lanes, row pairs
    } else {
      v32 = (uint32_t)v;
#pragma unroll
      for (int m = 0; m < Ls - 1; m++) v32 = add4_32(v32, __shfl_xor_sync(0xffffffffu, v32, 1 << m));
    }
    __syncthreads();   // sub[] cleared
    const int cov_rows = H - ty * TILE;                    // rows of this tile inside the image
    const int cov_cols = W - x0;
    // unrolled over the six levels: sizes, masks and store widths are constants per level
#pragma unroll
    for (int L = 1; L <= 6; L++) {
      if (L < Ls) continue;                                // entries stay 0 (sub[] cleared)
      uint64_t ang;
      if (L == 1) {
        ang = v;                                           // (Ls == 1 here; rows summed above)
      } else {
        if (L == 2 && Ls == 1) v32 = (uint32_t)pair4(v);     // 32 lanes -> 16
        else if (L > Ls) v32 = pair4_32(v32);              // widen the columns
        if (L <= 5) {
          v32 = add4_32(v32, __shfl_xor_sync(0xffffffffu, v32, 1 << (L - 1)));   // and the rows
        } else {
          if (lane == 0) l6_part[warp] = v32;
          __syncthreads();
          v32 = add4_32((uint32_t)l6_part[0], (uint32_t)l6_part[1]);
        }
        ang = v32;
      }
      const int nb = TILE >> L;                              // blocks per side at this level
      const int br = r >> L;
      if ((r & ((1 << L) - 1)) == 0) {
        // angle 0 for levels below lmin and for blocks not entirely inside the image
        const bool row_cov = (br + 1) * (1 << L) <= cov_rows;
        int ncol = cov_cols >> L;
        if (ncol > nb) ncol = nb;
        if (L < lmin || !row_cov || ncol <= 0) ang = 0;
        else if (ncol < nb) ang &= (1ull << (2 * ncol)) - 1ull;
        // one block row = 2 nb bits at byte subtree_off(L) + br * nb / 4
        if (L == 1) *reinterpret_cast<uint64_t*>(sub + br * 8) = ang;
        else if (L == 2) *reinterpret_cast<uint32_t*>(sub + subtree_off(2) + br * 4) = (uint32_t)ang;
        else if (L == 3) *reinterpret_cast<uint16_t*>(sub + subtree_off(3) + br * 2) = (uint16_t)ang;
        else if (L == 4) sub[subtree_off(4) + br] = (uint8_t)ang;
        else {
          const int off = subtree_off(L) * 8 + br * 2 * nb;   // 4 or 2 bits: shared bytes, OR-ed in
          atomicOr(reinterpret_cast<unsigned int*>(sub) + (off >> 5),
                   (uint32_t)(ang & ((1u << (2 * nb)) - 1)) << (off & 31));
        }
      }
      if (L == 6 && r == 0) B.sigma6[g] = (uint8_t)(v32 & 3u);  // raw tile sum for the top levels
    }
  };
  const int ls_rt = lmin < 1 ? 1 : (lmin > 4 ? 4 : lmin);   // uniform over the CTA (one tile)
  if (ls_rt == 1) levels(LevelTag<1>());
  else if (ls_rt == 2) levels(LevelTag<2>());
  else if (ls_rt == 3) levels(LevelTag<3>());
  else levels(LevelTag<4>());
  __syncthreads();
  // subtree to global (352 bytes)
  {
    const uint32_t* s32 = reinterpret_cast<const uint32_t*>(sub);
    uint32_t* g32 = reinterpret_cast<uint32_t*>(B.subtree + (size_t)g * SUBTREE_BYTES);
    for (int i = r; i < SUBTREE_BYTES / 4; i += 64) g32[i] = s32[i];
  }
  if (MODE == MODE_ENC && r < 8) {
    const uint32_t zc = zero_cnt[0][r] + zero_cnt[1][r];
    atomicAdd(B.hist_acc + 16 * img + r, zc);
    if (B.tile_cnt) B.tile_cnt[8 * (size_t)g + r] = (uint16_t)zc;   // label-0 pixels of this tile for b = r + 1
  }
  if (MODE == MODE_DEC && r == 0 && B.tile_cnt) B.tile_cnt[8 * (size_t)g] = (uint16_t)(zero_cnt[0][0] + zero_cnt[1][0]);
}

// The workspace's zero region (error word, tickets, counters, flags), cleared at the
// start of every operation by a kernel rather than a memset, so that the chain of
// programmatically dependent launches runs on from the previous operation.
__global__ void __launch_bounds__(256) k_zero(uint4* p, uint32_t n16) {
  pdl_wait();      // the previous kernel may still use this workspace
  pdl_trigger();
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += gridDim.x * blockDim.x)
    p[i] = make_uint4(0u, 0u, 0u, 0u);
}
cudaError_t launch_zero(void* p, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return cudaSuccess;
  if ((reinterpret_cast<uintptr_t>(p) & 15) || (bytes & 15)) return cudaMemsetAsync(p, 0, bytes, st);
  const uint32_t n16 = (uint32_t)(bytes / 16);
  uint32_t grid = (n16 + 255) / 256;
  if (grid > 1216) grid = 1216;
  return launch_pdl(k_zero, dim3(grid), dim3(256), 0, st, reinterpret_cast<uint4*>(p), n16);
}

// general = some image has W % 64 != 0 or a ragged tile row (rows that straddle blocks)
void launch_pass1(const Batch& B, int mode, bool general, bool any_med, cudaStream_t st) {
  if (B.total_tiles == 0) return;
  if (mode == MODE_ENC) {
    if (any_med) {
      if (general) launch_pdl(k_pass1<MODE_ENC, true, true>, dim3(B.total_tiles), dim3(64), 0, st, B);
      else launch_pdl(k_pass1<MODE_ENC, false, true>, dim3(B.total_tiles), dim3(64), 0, st, B);
    } else {
      if (general) launch_pdl(k_pass1<MODE_ENC, true, false>, dim3(B.total_tiles), dim3(64), 0, st, B);
      else launch_pdl(k_pass1<MODE_ENC, false, false>, dim3(B.total_tiles), dim3(64), 0, st, B);
    }
  } else {
    if (general) launch_pdl(k_pass1<MODE_DEC, true, false>, dim3(B.total_tiles), dim3(64), 0, st, B);
    else launch_pdl(k_pass1<MODE_DEC, false, false>, dim3(B.total_tiles), dim3(64), 0, st, B);
  }
}

}  // namespace rdhei
