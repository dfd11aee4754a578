// decode.cu -- K1 receiver's second pass (Sec. III-A-3 "receiver has only K1",
// Sec. III-B-3; Eq. roration2): de-rotate the decrypted image held in the stash and
// restore the replaced MSBs from the last label-1 pixel to the left.
//
// The restoration only looks left along a row (omega glide), so the tiles of a
// 64-row strip depend on each other from left to right and strips are independent.
// One CTA walks one strip: per tile it gathers the rotated tile (micro-block
// de-rotation, permute.cuh), restores the fields inside the tile, and carries, per
// row, the field of the last label-1 pixel into the next tile.  The next tile's
// data is fetched into registers while the current one is processed.
#include "permute.cuh"
#include "../../include/rdhei.h"

namespace rdhei {

// Byte-permute selector for a word whose label-1 bytes form the pattern z (bit k = byte
// k): result byte j takes byte j' of the word, j' the last label-1 byte at or before j,
// or byte 4 (the carried field) when bytes 0..j are all label 0.
__host__ __device__ __forceinline__ uint32_t fill_selector(uint32_t z) {
  uint32_t sel = 0, src = 4;
  for (int j = 0; j < 4; j++) {
    if ((z >> j) & 1u) src = (uint32_t)j;
    sel |= src << (4 * j);
  }
  return sel;
}

template <bool ANY_LMR, bool ANY_MED>
__global__ void __launch_bounds__(256, 6) k_dec_strip(Batch B) {
  pdl_wait();      // the previous kernel of the operation has finished
  pdl_trigger();
  __shared__ __align__(16) uint8_t tin[TILE * TPITCH];
  __shared__ __align__(16) uint8_t ain[TILE * TPITCH];
  __shared__ __align__(16) uint8_t tout[TILE * TPITCH];
  __shared__ __align__(16) uint8_t aout[TILE * TPITCH];
  __shared__ __align__(16) uint8_t sub[SUBTREE_BYTES];
  __shared__ uint32_t selt[16];
  __shared__ uint8_t rowcarry[TILE];
  __shared__ uint32_t fillsel[16];

  const int t = threadIdx.x;
  const uint32_t s = blockIdx.x;
  const int img = (int)__ldg(B.strip_owner + s);
  const ImgDesc& d = B.desc[img];
  const int H = d.H, W = d.W;
  const rdhei_info* info = reinterpret_cast<const rdhei_info*>(d.info);
  const int b = d.b > 0 ? d.b : info->b;
  const bool lmr = ANY_LMR && d.variant == RDHEI_LMR;
  const bool med = ANY_MED && d.med != 0;
  const uint32_t ty = s - __ldg(B.strip_prefix + img);
  const uint32_t tiles_x = d.tiles_x;
  // the replaced field: EMR top b bits, LMR bits 6 .. 8-b (Sec. III-B-2)
  const uint32_t FM = lmr ? (((1u << (b - 1)) - 1u) << (8 - b)) : ((0xFFu << (8 - b)) & 0xFFu);
  const uint32_t FM4 = FM * 0x01010101u;
  const int row = tile_row_of(t), quarter = t & 3;
  const int y = (int)ty * TILE + row;
  if (t < 16) selt[t] = pair_selectors((4u - (t & 3u)) & 3u, (4u - (t >> 2)) & 3u);   // inverse 2x2 turns
  if (t >= 16 && t < 32) fillsel[t - 16] = fill_selector(t - 16);

  // rotated tile of original tile (ty, tx): my 16 bytes of the stash and 16 aux bits
  uint32_t nw[4], na = 0, nU = 0;
  auto fetch = [&](uint32_t tx) {
    const uint32_t g = d.tile_base + ty * tiles_x + tx;
    const TileMap tm = B.tilemap[g];
    nU = tm.dec_shi;
    const uint32_t Q = tm.dec_dst;
    const bool q_ok = RDHEI_IDX_OK(B.err, Q < tiles_x * d.tiles_y);
    const int qy = (int)(Q / tiles_x) * TILE + row, qx = (int)(Q % tiles_x) * TILE + 16 * quarter;
    int valid = (q_ok && qy < H) ? min(16, W - qx) : 0;
    if (valid < 0) valid = 0;
    const uint8_t* sp = d.stash + (size_t)qy * W + qx;
    if (valid == 16 && ((reinterpret_cast<uintptr_t>(sp) & 15) == 0)) {
      const uint4 v = *reinterpret_cast<const uint4*>(sp);
      nw[0] = v.x; nw[1] = v.y; nw[2] = v.z; nw[3] = v.w;
    } else {
#pragma unroll
      for (int i = 0; i < 4; i++) {
        uint32_t v = 0;
#pragma unroll
        for (int k = 0; k < 4; k++)
          if (4 * i + k < valid) v |= (uint32_t)sp[4 * i + k] << (8 * k);
        nw[i] = v;
      }
    }
    const uint16_t* ap = reinterpret_cast<const uint16_t*>(B.aux + (size_t)(d.tile_base + Q) * AUX_BYTES);
    na = q_ok ? ap[row * 4 + quarter] : 0u;
  };
  fetch(0);

  for (uint32_t tx = 0; tx < tiles_x; tx++) {
    const uint32_t P = ty * tiles_x + tx;
    const uint32_t U = nU;
    // 1. the fetched tile and its aux plane into shared memory, the subtree of P
    *reinterpret_cast<uint4*>(skewed_chunk<true>(tin, row, quarter)) = make_uint4(nw[0], nw[1], nw[2], nw[3]);
    {
      uint32_t e[4];
#pragma unroll
      for (int i = 0; i < 4; i++) e[i] = (((na >> (4 * i)) & 0xFu) * 0x00204081u) & 0x01010101u;
      *reinterpret_cast<uint4*>(skewed_chunk<true>(ain, row, quarter)) = make_uint4(e[0], e[1], e[2], e[3]);
    }
    if (t < SUBTREE_BYTES / 4)
      reinterpret_cast<uint32_t*>(sub)[t] =
          __ldg(reinterpret_cast<const uint32_t*>(B.subtree + (size_t)(d.tile_base + P) * SUBTREE_BYTES) + t);
    if (tx + 1 < tiles_x) fetch(tx + 1);        // in flight while this tile is processed
    __syncthreads();

    // 2. de-rotation: original micro-block (mr, mc) <- rotated micro-block (qr, qc)
    {
      const uint32_t mr = t >> 4, mc = t & 15;
      uint32_t qr, qc, S1;
      dec_microblock_src(sub, U, mr, mc, qr, qc, S1);
      const uint32_t nib = sub_level1_nibbles(sub, mr, mc);
      const uint32_t sT = selt[nib & 0xF], sB = selt[nib >> 4];
      const uint32_t inv = (4u - S1) & 3u;
      uint32_t w0, w1, w2, w3;
      ld_micro_skewed<true>(tin, qr, qc, w0, w1, w2, w3);
      turn4x4(w0, w1, w2, w3, inv);
      turn_subblocks(w0, w1, w2, w3, sT, sB);
      st_micro(tout, mr, mc, w0, w1, w2, w3);
      ld_micro_skewed<true>(ain, qr, qc, w0, w1, w2, w3);
      turn4x4(w0, w1, w2, w3, inv);
      turn_subblocks(w0, w1, w2, w3, sT, sB);
      st_micro(aout, mr, mc, w0, w1, w2, w3);
    }
    __syncthreads();

    // 3. labels and decrypted values of my 16 pixels
    const int x = (int)tx * TILE + 16 * quarter;
    int valid = (y < H) ? min(16, W - x) : 0;
    if (valid < 0) valid = 0;
    uint32_t v[4], lw[4];
    {
      const uint4 v4 = *reinterpret_cast<const uint4*>(tout + row * TPITCH + 16 * quarter);
      const uint4 a4 = *reinterpret_cast<const uint4*>(aout + row * TPITCH + 16 * quarter);
      const uint32_t vv[4] = {v4.x, v4.y, v4.z, v4.w}, aa[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
      for (int i = 0; i < 4; i++) {
        if (lmr) {
          lw[i] = (vv[i] >> 7) & 0x01010101u;
          v[i] = (vv[i] & 0x7F7F7F7Fu) | (aa[i] << 7);            // bit 7 := eta
        } else {
          lw[i] = vv[i] & 0x01010101u;
          v[i] = vv[i] ^ aa[i];                                   // LSB := map XOR s (decrypted LSB)
        }
      }
      if (valid < 16) {
#pragma unroll
        for (int i = 0; i < 4; i++) {
          const int nv = valid - 4 * i;                           // pixels past the row end: label 0
          lw[i] &= nv <= 0 ? 0u : nv >= 4 ? 0xFFFFFFFFu : ((1u << (8 * nv)) - 1u);
        }
      }
      if (x == 0 && valid > 0 && !med) lw[0] |= 1u;              // first image column: non-redundant
    }
    if (ANY_MED && med) {
      // MED variant: the prediction needs recovered upper neighbours, so this pass only
      // writes the decrypted, de-rotated pixels and their labels; the wavefront kernel
      // restores the fields
      uint32_t bits16 = 0;
#pragma unroll
      for (int i = 0; i < 4; i++) bits16 |= ((((lw[i] & 0x01010101u) * 0x01020408u) >> 24) & 0xFu) << (4 * i);
      reinterpret_cast<uint16_t*>(B.lab + (size_t)(d.tile_base + P) * AUX_BYTES)[row * 4 + quarter] = (uint16_t)bits16;
      if (valid > 0) {
        uint8_t* dst = d.dst + (size_t)y * W + x;
        if (valid == 16 && ((reinterpret_cast<uintptr_t>(dst) & 15) == 0)) {
          *reinterpret_cast<uint4*>(dst) = make_uint4(v[0], v[1], v[2], v[3]);
        } else {
#pragma unroll
          for (int k = 0; k < 16; k++)
            if (k < valid) dst[k] = (uint8_t)(v[k >> 2] >> (8 * (k & 3)));
        }
      }
      __syncthreads();
      continue;
    }
    // 4. the field of the last label-1 pixel among my 16, then the carry into them: the
    //    last such field of the quarters to my left, else the strip's carry from the
    //    previous tile
    uint32_t zw[4];                                               // label pattern per word, bit k = byte k
#pragma unroll
    for (int i = 0; i < 4; i++) zw[i] = (lw[i] * 0x01020408u) >> 24;
    const uint32_t pat = zw[0] | (zw[1] << 4) | (zw[2] << 8) | (zw[3] << 12);
    const uint32_t has = pat != 0u;
    uint32_t fld = 0;
    {
      const uint32_t lb = 31u - (uint32_t)__clz(pat | 1u);       // last label-1 byte (when has)
      const uint32_t w01 = (lb & 4u) ? v[1] : v[0], w23 = (lb & 4u) ? v[3] : v[2];
      const uint32_t w = (lb & 8u) ? w23 : w01;
      if (has) fld = (w >> (8u * (lb & 3u))) & FM;
    }
    uint32_t ch = has, cf = fld;   // inclusive scan across the row's 4 lanes, "last one wins"
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
      const uint32_t oh = __shfl_up_sync(0xffffffffu, ch, o, 4), of = __shfl_up_sync(0xffffffffu, cf, o, 4);
      if (quarter >= o && !ch) { ch = oh; cf = of; }
    }
    uint32_t in_has = __shfl_up_sync(0xffffffffu, ch, 1, 4), in_fld = __shfl_up_sync(0xffffffffu, cf, 1, 4);
    if (quarter == 0) in_has = 0;
    if (!in_has) in_fld = tx > 0 ? rowcarry[row] : 0u;
    __syncwarp();
    if (quarter == 3 && ch) rowcarry[row] = (uint8_t)cf;      // carry into the next tile

    // 5. restore and store: per word one byte permute gives every byte the field of the
    //    last label-1 byte at or before it (selector table by label pattern), or the
    //    carried field (the second operand) when there is none
    if (valid > 0) {
      uint32_t carry4 = in_fld * 0x01010101u;
#pragma unroll
      for (int i = 0; i < 4; i++) {
        const uint32_t f = __byte_perm(v[i] & FM4, carry4, fillsel[zw[i]]);
        v[i] = (v[i] & ~FM4) | f;
        carry4 = __byte_perm(f, 0u, 0x3333u);
      }
      uint8_t* dst = d.dst + (size_t)y * W + x;
      if (valid == 16 && ((reinterpret_cast<uintptr_t>(dst) & 15) == 0)) {
        *reinterpret_cast<uint4*>(dst) = make_uint4(v[0], v[1], v[2], v[3]);
      } else {
#pragma unroll
        for (int k = 0; k < 16; k++)
          if (k < valid) dst[k] = (uint8_t)(v[k >> 2] >> (8 * (k & 3)));
      }
    }
    __syncthreads();   // shared tiles are rewritten by the next iteration
  }
}

void launch_dec_pass2(const Batch& B, bool any_lmr, bool any_med, cudaStream_t st) {
  if (B.total_strips == 0) return;
  if (any_med) {
    if (any_lmr) launch_pdl(k_dec_strip<true, true>, dim3(B.total_strips), dim3(256), 0, st, B);
    else launch_pdl(k_dec_strip<false, true>, dim3(B.total_strips), dim3(256), 0, st, B);
  } else {
    if (any_lmr) launch_pdl(k_dec_strip<true, false>, dim3(B.total_strips), dim3(256), 0, st, B);
    else launch_pdl(k_dec_strip<false, false>, dim3(B.total_strips), dim3(256), 0, st, B);
  }
}

}  // namespace rdhei
