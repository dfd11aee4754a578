// permute.cuh -- the in-tile part of the multi-scale block rotation (Eqs. roration,
// roration2) as a gather over 4 x 4 micro-blocks.
//
// A level-L quarter-turn moves a pixel inside its 2^L block as (u, v) -> (B-1-v, u):
// it acts on every coordinate bit below L on its own and leaves the bits >= L (which
// name the enclosing blocks) alone.  Composing the levels, bit j of a pixel's
// destination is bit j of its source turned by S_j, the sum of the angles of the
// source's enclosing blocks at the levels above j.  Inside a 64 x 64 tile this gives:
//   * micro-block (bits 5..2) destination: four table steps per 16 pixels;
//   * micro-block contents: each 2 x 2 sub-block turned by its own level-1 angle,
//     then the whole 4 x 4 turned by S_1 -- both done on four 32-bit rows with PRMT.
#pragma once
#include "common.cuh"

namespace rdhei {

constexpr int TPITCH = 80;   // shared-memory row pitch of a 64-byte tile row (bank spread)

// Tile row of thread t in the encode gather (256 threads, four per row; the row's
// quarters are four consecutive lanes).  A warp's 16-byte shared accesses of tile rows
// run in four phases of eight lanes, and with the 80-byte pitch two adjacent rows share
// four of their sixteen banks; so the lanes of a phase take rows r and r + 4 (80 words
// apart, disjoint banks) instead of r and r + 1.  Measured on 1000 x 512^2: the owner's
// gather 0.252 -> 0.241 ms; the decode gather 0.258 -> 0.254 ms together with the chunk
// skew below (alone it measured slower there, 0.266 ms).
__device__ __forceinline__ int tile_row_of(int t) {
  const int lane = t & 31;
  return 8 * (t >> 5) + ((lane >> 3) & 3) + 4 * ((lane >> 2) & 1);
}

// 2-bit angle of block (br, bc) at level L (1..6) from a tile's packed subtree.
__device__ __forceinline__ uint32_t sub_angle(const uint8_t* sub, int L, uint32_t br, uint32_t bc) {
  uint32_t e = br * (uint32_t)(TILE >> L) + bc;
  return (sub[subtree_off(L) + (e >> 2)] >> (2 * (e & 3))) & 3u;
}

// Level-1 angles of the four 2x2 sub-blocks of micro-block (mr, mc): low nibble =
// top sub-blocks (left angle bits 0-1, right bits 2-3), high nibble = bottom ones.
__device__ __forceinline__ uint32_t sub_level1_nibbles(const uint8_t* sub, uint32_t mr, uint32_t mc) {
  uint32_t e0 = (2 * mr) * 32 + 2 * mc;          // even entry -> nibble aligned
  uint32_t e1 = e0 + 32;
  uint32_t top = (sub[e0 >> 2] >> (2 * (e0 & 3))) & 0xFu;
  uint32_t bot = (sub[e1 >> 2] >> (2 * (e1 & 3))) & 0xFu;
  return top | (bot << 4);
}

// PRMT selectors turning the two 2x2 sub-blocks held in rows (w0, w1) by angles
// aL (columns 0-1) and aR (columns 2-3).  Row selectors per angle (bytes 0-3 of w0,
// 4-7 of w1): row 0 {0x10, 0x51, 0x45, 0x04}, row 1 {0x54, 0x40, 0x01, 0x15}.
__host__ __device__ __forceinline__ uint32_t pair_selectors(uint32_t aL, uint32_t aR) {
  const uint32_t R0 = 0x04455110u, R1 = 0x15014054u;
  uint32_t s0 = ((R0 >> (8 * aL)) & 0xFFu) | ((((R0 >> (8 * aR)) & 0xFFu) + 0x22u) << 8);
  uint32_t s1 = ((R1 >> (8 * aL)) & 0xFFu) | ((((R1 >> (8 * aR)) & 0xFFu) + 0x22u) << 8);
  return s0 | (s1 << 16);
}

// Quarter-turns (counter-clockwise, numpy.rot90 sense) of a 4x4 byte block held as
// four rows: new(i, j) = old(j, 3 - i) per turn.  Branch-free in `a`.
__device__ __forceinline__ void turn4x4(uint32_t& w0, uint32_t& w1, uint32_t& w2, uint32_t& w3, uint32_t a) {
  a &= 3u;
  uint32_t t0 = __byte_perm(w0, w1, 0x5140), t1 = __byte_perm(w0, w1, 0x7362);
  uint32_t t2 = __byte_perm(w2, w3, 0x5140), t3 = __byte_perm(w2, w3, 0x7362);
  uint32_t T0 = __byte_perm(t0, t2, 0x5410), T1 = __byte_perm(t0, t2, 0x7632);
  uint32_t T2 = __byte_perm(t1, t3, 0x5410), T3 = __byte_perm(t1, t3, 0x7632);
  const bool odd = a & 1u;
  uint32_t x0 = odd ? T0 : w0, x1 = odd ? T1 : w1, x2 = odd ? T2 : w2, x3 = odd ? T3 : w3;
  const bool rr = ((a ^ (a >> 1)) & 1u) != 0;     // a == 1 or 2: reverse the row order
  uint32_t y0 = rr ? x3 : x0, y1 = rr ? x2 : x1, y2 = rr ? x1 : x2, y3 = rr ? x0 : x3;
  const uint32_t sel = (a & 2u) ? 0x0123u : 0x3210u;   // a == 2 or 3: reverse each row
  w0 = __byte_perm(y0, 0, sel); w1 = __byte_perm(y1, 0, sel);
  w2 = __byte_perm(y2, 0, sel); w3 = __byte_perm(y3, 0, sel);
}

// Turn the four 2x2 sub-blocks of a 4x4 block; `selTop` / `selBot` from pair_selectors.
__device__ __forceinline__ void turn_subblocks(uint32_t& w0, uint32_t& w1, uint32_t& w2, uint32_t& w3,
                                               uint32_t selTop, uint32_t selBot) {
  uint32_t n0 = __byte_perm(w0, w1, selTop & 0xFFFFu), n1 = __byte_perm(w0, w1, selTop >> 16);
  uint32_t n2 = __byte_perm(w2, w3, selBot & 0xFFFFu), n3 = __byte_perm(w2, w3, selBot >> 16);
  w0 = n0; w1 = n1; w2 = n2; w3 = n3;
}

// Source micro-block of output micro-block (mr, mc) for the ENCODE gather, and S_1.
// U = sum of the angles above level 6 enclosing the source tile.
__device__ __forceinline__ void enc_microblock_src(const uint8_t* sub, uint32_t U, uint32_t mr, uint32_t mc,
                                                   uint32_t& pr, uint32_t& pc, uint32_t& S1) {
  uint32_t S = U + sub_angle(sub, 6, 0, 0);
  pr = 0; pc = 0;
#pragma unroll
  for (int j = 5; j >= 2; --j) {
    uint32_t qb = (((mr >> (j - 2)) & 1u) << 1) | ((mc >> (j - 2)) & 1u);
    uint32_t pb = rot_bits(ROT_INV_LUT, S, qb);
    pr = (pr << 1) | (pb >> 1);
    pc = (pc << 1) | (pb & 1u);
    S += sub_angle(sub, j, pr, pc);
  }
  S1 = S & 3u;
}

// Rotated-domain micro-block holding original micro-block (mr, mc) (DECODE), and S_1.
__device__ __forceinline__ void dec_microblock_src(const uint8_t* sub, uint32_t U, uint32_t mr, uint32_t mc,
                                                   uint32_t& qr, uint32_t& qc, uint32_t& S1) {
  uint32_t S = U + sub_angle(sub, 6, 0, 0);
  qr = 0; qc = 0;
#pragma unroll
  for (int j = 5; j >= 2; --j) {
    uint32_t pb = (((mr >> (j - 2)) & 1u) << 1) | ((mc >> (j - 2)) & 1u);
    uint32_t qb = rot_bits(ROT_FWD_LUT, S, pb);
    qr = (qr << 1) | (qb >> 1);
    qc = (qc << 1) | (qb & 1u);
    S += sub_angle(sub, j, mr >> (j - 2), mc >> (j - 2));
  }
  S1 = S & 3u;
}

__device__ __forceinline__ void ld_micro(const uint8_t* t, uint32_t r, uint32_t c, uint32_t& w0, uint32_t& w1,
                                         uint32_t& w2, uint32_t& w3) {
  const uint8_t* p = t + (4 * r) * TPITCH + 4 * c;
  w0 = *reinterpret_cast<const uint32_t*>(p);
  w1 = *reinterpret_cast<const uint32_t*>(p + TPITCH);
  w2 = *reinterpret_cast<const uint32_t*>(p + 2 * TPITCH);
  w3 = *reinterpret_cast<const uint32_t*>(p + 3 * TPITCH);
}
__device__ __forceinline__ void st_micro(uint8_t* t, uint32_t r, uint32_t c, uint32_t w0, uint32_t w1,
                                         uint32_t w2, uint32_t w3) {
  uint8_t* p = t + (4 * r) * TPITCH + 4 * c;
  *reinterpret_cast<uint32_t*>(p) = w0;
  *reinterpret_cast<uint32_t*>(p + TPITCH) = w1;
  *reinterpret_cast<uint32_t*>(p + 2 * TPITCH) = w2;
  *reinterpret_cast<uint32_t*>(p + 3 * TPITCH) = w3;
}

// The encode gather's source tile and label plane in shared memory: the four 16-byte
// chunks of row R are rotated by (R >> 3) & 3 places.  The rotation reads source
// micro-blocks at permuted positions -- a whole column of them when the tile turns by
// an odd angle -- and with the 80-byte pitch a micro-block column falls on only four
// banks; the skew spreads it (3.3 -> 2.2 wavefronts per micro-block row read on
// average, by a bank model over random angles; the fused encode kernel measured
// 0.486 -> 0.483 ms on 1000 x 512^2).
// SKEW = false gives the plain layout (the separable gather: the skew's address
// arithmetic costs it a spill at its 40-register bound and measured slower there).
template <bool SKEW, typename T>
__device__ __forceinline__ T* skewed_chunk(T* t, int row, int q) {
  return t + row * TPITCH + 16 * (SKEW ? ((q + (row >> 3)) & 3) : q);
}
template <bool SKEW>
__device__ __forceinline__ void ld_micro_skewed(const uint8_t* t, uint32_t r, uint32_t c, uint32_t& w0,
                                                uint32_t& w1, uint32_t& w2, uint32_t& w3) {
  // rows 4r .. 4r + 3 share (row >> 3) = r >> 1
  const uint8_t* p = t + (4 * r) * TPITCH + 16 * (SKEW ? (((c >> 2) + (r >> 1)) & 3u) : (c >> 2)) + 4 * (c & 3u);
  w0 = *reinterpret_cast<const uint32_t*>(p);
  w1 = *reinterpret_cast<const uint32_t*>(p + TPITCH);
  w2 = *reinterpret_cast<const uint32_t*>(p + 2 * TPITCH);
  w3 = *reinterpret_cast<const uint32_t*>(p + 3 * TPITCH);
}

// 16 per-pixel flags (one byte each, flag bit `bit`) of a 16-byte row chunk ->
// 16 bits MSB-first (bit 15 = first pixel).
__device__ __forceinline__ uint32_t flags16(const uint32_t w[4], int bit) {
  uint32_t v = 0;
#pragma unroll
  for (int i = 0; i < 4; i++) {
    // the multiply gathers the word's four flags into bits 31..28 (pixel 4i at bit 31;
    // no two partial products share a bit), then they are shifted into v
    const uint32_t x = ((w[i] >> bit) & 0x01010101u) * 0x80402010u;
    v = __funnelshift_l(x, v, 4);
  }
  return v & 0xFFFFu;
}

// Write `n` (<= 16) MSB-first bits v16 (bit 15 first) at stream bit `pos`.  `plain`:
// the caller guarantees pos % 16 == 0 and n == 16 for every chunk of the stream (a
// plain 16-bit store); otherwise bits are OR-ed into words the launcher zeroed.
__device__ __forceinline__ void put_bits16(uint8_t* stream, uint32_t pos, uint32_t v16, int n, bool plain) {
  if (n <= 0) return;
  if (plain) {
    *reinterpret_cast<uint16_t*>(stream + (pos >> 3)) = (uint16_t)(((v16 >> 8) & 0xFFu) | ((v16 & 0xFFu) << 8));
    return;
  }
  v16 &= (0xFFFFu << (16 - n)) & 0xFFFFu;
  uint32_t* w = reinterpret_cast<uint32_t*>(stream);
  const uint32_t wi = pos >> 5;
  const uint32_t sh = pos & 31;
  uint64_t run = ((uint64_t)v16 << 48) >> sh;              // bit 63 = word wi's first bit
  uint32_t hi = (uint32_t)(run >> 32), lo = (uint32_t)run;
  if (hi) atomicOr(w + wi, bswap32(hi));
  if (lo) atomicOr(w + wi + 1, bswap32(lo));
}

}  // namespace rdhei
