// decode.cu -- K1 receiver's second pass (Sec. III-A-3 "receiver has only K1",
// Sec. III-B-3; Eq. roration2): de-rotate the decrypted image held in the stash and
// restore the replaced MSBs from the last label-1 pixel to the left.
//
// The restoration only looks left along a row (omega glide), so tile (r, c) depends
// on tile (r, c - 1) only.  Tiles are taken in ticket order (row-major per image) and
// hand the per-row carry ("field of the last label-1 pixel so far") to their right
// neighbour with a decoupled look-back: each tile publishes its own row aggregates
// at once and its inclusive carries once its left neighbour's are known.
#include "permute.cuh"
#include "../../include/rdhei.h"

namespace rdhei {

constexpr uint32_t FLAG_AGG = 1, FLAG_INC = 2;
constexpr int TK_DEC = 0;

template <bool ANY_LMR>
__global__ void __launch_bounds__(256) k_dec_pass2(Batch B) {
  __shared__ __align__(16) uint8_t tin[TILE * TPITCH];
  __shared__ __align__(16) uint8_t ain[TILE * TPITCH];
  __shared__ __align__(16) uint8_t tout[TILE * TPITCH];
  __shared__ __align__(16) uint8_t aout[TILE * TPITCH];
  __shared__ __align__(16) uint8_t sub[SUBTREE_BYTES];
  __shared__ uint32_t selt[16];
  __shared__ uint8_t rowcarry[TILE];
  __shared__ uint32_t s_ticket;

  const int t = threadIdx.x;
  if (t == 0) s_ticket = atomicAdd(B.tickets + TK_DEC, 1u);
  __syncthreads();
  const uint32_t g = s_ticket;
  const int img = owner_of(B.tile_prefix, B.n_images, g);
  const ImgDesc& d = B.desc[img];
  const int H = d.H, W = d.W;
  const rdhei_info* info = reinterpret_cast<const rdhei_info*>(d.info);
  const int b = d.b > 0 ? d.b : info->b;
  const bool lmr = ANY_LMR && d.variant == RDHEI_LMR;
  const uint32_t P = g - d.tile_base;
  const int ptx = (int)(P % d.tiles_x);
  const int py0 = (int)(P / d.tiles_x) * TILE, px0 = ptx * TILE;
  const TileMap tm = B.tilemap[g];
  const uint32_t Q = tm.dec_dst, U = tm.dec_shi;
  const int qy0 = (int)(Q / d.tiles_x) * TILE, qx0 = (int)(Q % d.tiles_x) * TILE;
  // the replaced field: EMR top b bits, LMR bits 6 .. 8-b (Sec. III-B-2)
  const uint32_t FM = lmr ? (((1u << (b - 1)) - 1u) << (8 - b)) : ((0xFFu << (8 - b)) & 0xFFu);

  {
    const uint32_t* s32 = reinterpret_cast<const uint32_t*>(B.subtree + (size_t)(d.tile_base + P) * SUBTREE_BYTES);
    if (t < SUBTREE_BYTES / 4) reinterpret_cast<uint32_t*>(sub)[t] = __ldg(s32 + t);
    // inverse turns of the 2x2 sub-blocks
    if (t < 16) selt[t] = pair_selectors((4u - (t & 3u)) & 3u, (4u - (t >> 2)) & 3u);
  }

  const int row = t >> 2, quarter = t & 3;
  // 1. load the decrypted tile Q from the stash, and its aux plane
  {
    const int y = qy0 + row, x = qx0 + 16 * quarter;
    int valid = (y < H) ? min(16, W - x) : 0;
    if (valid < 0) valid = 0;
    const uint8_t* s = d.stash + (size_t)y * W + x;
    uint32_t w[4];
    if (valid == 16 && ((reinterpret_cast<uintptr_t>(s) & 15) == 0)) {
      uint4 v = *reinterpret_cast<const uint4*>(s);
      w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
    } else {
#pragma unroll
      for (int i = 0; i < 4; i++) {
        uint32_t v = 0;
#pragma unroll
        for (int k = 0; k < 4; k++)
          if (4 * i + k < valid) v |= (uint32_t)s[4 * i + k] << (8 * k);
        w[i] = v;
      }
    }
    *reinterpret_cast<uint4*>(tin + row * TPITCH + 16 * quarter) = make_uint4(w[0], w[1], w[2], w[3]);
    const uint64_t arow = reinterpret_cast<const uint64_t*>(B.aux + (size_t)(d.tile_base + Q) * AUX_BYTES)[row];
    const uint32_t a16 = (uint32_t)(arow >> (16 * quarter)) & 0xFFFFu;
    uint32_t e[4];
#pragma unroll
    for (int i = 0; i < 4; i++) e[i] = (((a16 >> (4 * i)) & 0xFu) * 0x00204081u) & 0x01010101u;
    *reinterpret_cast<uint4*>(ain + row * TPITCH + 16 * quarter) = make_uint4(e[0], e[1], e[2], e[3]);
  }
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
    ld_micro(tin, qr, qc, w0, w1, w2, w3);
    turn4x4(w0, w1, w2, w3, inv);
    turn_subblocks(w0, w1, w2, w3, sT, sB);
    st_micro(tout, mr, mc, w0, w1, w2, w3);
    ld_micro(ain, qr, qc, w0, w1, w2, w3);
    turn4x4(w0, w1, w2, w3, inv);
    turn_subblocks(w0, w1, w2, w3, sT, sB);
    st_micro(aout, mr, mc, w0, w1, w2, w3);
  }
  __syncthreads();

  // 3. labels and decrypted values in the original frame
  const int y = py0 + row, x = px0 + 16 * quarter;
  int valid = (y < H) ? min(16, W - x) : 0;
  if (valid < 0) valid = 0;
  uint32_t v[4], lab[4];
  {
    const uint4 v4 = *reinterpret_cast<const uint4*>(tout + row * TPITCH + 16 * quarter);
    const uint4 a4 = *reinterpret_cast<const uint4*>(aout + row * TPITCH + 16 * quarter);
    const uint32_t vv[4] = {v4.x, v4.y, v4.z, v4.w}, aa[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
    for (int i = 0; i < 4; i++) {
      if (lmr) {
        lab[i] = (vv[i] >> 7) & 0x01010101u;
        v[i] = (vv[i] & 0x7F7F7F7Fu) | (aa[i] << 7);            // bit 7 := eta
      } else {
        lab[i] = vv[i] & 0x01010101u;
        v[i] = vv[i] ^ aa[i];                                   // LSB := map XOR s (decrypted LSB)
      }
      // pixels past the row end are never label 1
      int nv = valid - 4 * i;
      lab[i] &= nv <= 0 ? 0u : nv >= 4 ? 0xFFFFFFFFu : ((1u << (8 * nv)) - 1u);
    }
    if (x == 0 && valid > 0) lab[0] |= 1u;                      // first image column: non-redundant
  }
  // segment aggregate: field of the last label-1 pixel among my 16
  uint32_t has = 0, fld = 0;
#pragma unroll
  for (int i = 0; i < 16; i++) {
    const uint32_t li = (lab[i >> 2] >> (8 * (i & 3))) & 1u;
    const uint32_t fi = ((v[i >> 2] >> (8 * (i & 3))) & FM) >> (8 - b);
    if (li) { has = 1; fld = fi; }
  }
  // exclusive combine across the 4 quarters of the row (lanes 4k..4k+3)
  uint32_t in_has = 0, in_fld = 0;
  {
    uint32_t ch = has, cf = fld;   // inclusive scan, "last one wins"
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
      uint32_t oh = __shfl_up_sync(0xffffffffu, ch, o, 4), of = __shfl_up_sync(0xffffffffu, cf, o, 4);
      if (quarter >= o && !ch) { ch = oh; cf = of; }
    }
    in_has = __shfl_up_sync(0xffffffffu, ch, 1, 4);
    in_fld = __shfl_up_sync(0xffffffffu, cf, 1, 4);
    if (quarter == 0) { in_has = 0; in_fld = 0; }
    if (quarter == 3) {
      B.tile_rows[(size_t)g * 128 + row] = (uint8_t)((ch << 7) | cf);        // aggregate
      if (ptx == 0) B.tile_rows[(size_t)g * 128 + 64 + row] = (uint8_t)((ch << 7) | cf);
    }
  }
  __syncthreads();
  if (t == 0) {
    __threadfence();
    st_release_u32(B.tile_flags + g, ptx == 0 ? FLAG_INC : FLAG_AGG);
  }

  // 4. look-back for the carries entering this tile from the left
  if (ptx > 0) {
    if (t < 32) {
      uint32_t need = 3u;                       // rows t and t + 32 unresolved
      uint32_t c0 = 0, c1 = 0;
      uint32_t cur = g - 1;
      const uint64_t t0 = globaltimer_ns();
      bool timed_out = false;
      while (need) {
        uint32_t f = ld_acquire_u32(B.tile_flags + cur);
        if (f == 0) {
          if (globaltimer_ns() - t0 > WAIT_LIMIT_NS) { timed_out = true; break; }
          __nanosleep(32);
          continue;
        }
        const uint8_t* rv = B.tile_rows + (size_t)cur * 128 + (f == FLAG_INC ? 64 : 0);
        const uint32_t r0 = rv[t], r1 = rv[t + 32];
        if ((need & 1u) && (r0 >> 7)) { c0 = r0 & 0x7Fu; need &= ~1u; }
        if ((need & 2u) && (r1 >> 7)) { c1 = r1 & 0x7Fu; need &= ~2u; }
        if (f == FLAG_INC) need = 0;           // an inclusive value always has a label-1 pixel
        if (cur == d.tile_base) break;
        --cur;
      }
      if (timed_out) {
        set_error(B.err, ERR_TIMEOUT);
        const_cast<rdhei_info*>(info)->status = ERR_TIMEOUT;
      }
      rowcarry[t] = (uint8_t)c0;
      rowcarry[t + 32] = (uint8_t)c1;
    }
    __syncthreads();
    if (quarter == 3) {
      const uint32_t agg = B.tile_rows[(size_t)g * 128 + row];
      const uint32_t inc = (agg >> 7) ? agg : (0x80u | rowcarry[row]);
      B.tile_rows[(size_t)g * 128 + 64 + row] = (uint8_t)inc;
    }
    __syncthreads();
    if (t == 0) {
      __threadfence();
      st_release_u32(B.tile_flags + g, FLAG_INC);
    }
    if (!in_has) { in_has = 1; in_fld = rowcarry[row]; }
  }

  // 5. restore: label-0 pixels take the field of the last label-1 pixel to their left
  if (valid > 0) {
    uint32_t c = in_fld << (8 - b);
#pragma unroll
    for (int i = 0; i < 4; i++) {
      uint32_t o = v[i];
#pragma unroll
      for (int k = 0; k < 4; k++) {
        const uint32_t sh = 8 * k;
        if ((lab[i] >> sh) & 1u) c = (o >> sh) & FM;
        else o = (o & ~(FM << sh)) | (c << sh);
      }
      v[i] = o;
    }
    uint8_t* dst = d.dst + (size_t)y * W + x;
    if (valid == 16 && ((reinterpret_cast<uintptr_t>(dst) & 15) == 0)) {
      *reinterpret_cast<uint4*>(dst) = make_uint4(v[0], v[1], v[2], v[3]);
    } else {
      for (int k = 0; k < valid; k++) dst[k] = (uint8_t)(v[k >> 2] >> (8 * (k & 3)));
    }
  }
}

void launch_dec_pass2(const Batch& B, bool any_lmr, cudaStream_t st) {
  if (B.total_tiles == 0) return;
  if (any_lmr) k_dec_pass2<true><<<B.total_tiles, 256, 0, st>>>(B);
  else k_dec_pass2<false><<<B.total_tiles, 256, 0, st>>>(B);
}

}  // namespace rdhei
