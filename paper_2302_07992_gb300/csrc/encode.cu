// encode.cu -- content owner's second half: top rotation levels + choice of b
// (k_topmap) and the gather pass that labels, rotates, encrypts and embeds the map
// (k_enc_pass2).
#include "permute.cuh"
#include "../../include/rdhei.h"

namespace rdhei {

// Raw block sums (mod 4) for levels 7..n live in shared memory, row-major per level.
constexpr int TOP_SMEM = 11 * 1024;

__device__ __forceinline__ int top_off(int H, int W, int L) {
  int off = 0;
  for (int l = 7; l < L; l++) off += (H >> l) * (W >> l);
  return off;
}

// One CTA per image.
//   owner:    histogram -> hist[9], b (Eq. optimal_b), capacity, into rdhei_info;
//   both:     sums of the tile totals up the levels above 6 (Eq. roration) and, per
//             tile, where the composed rotation sends it and the angle sum above 6.
__global__ void __launch_bounds__(256) k_topmap(Batch B, int owner) {
  pdl_wait();      // the previous kernel of the operation has finished
  pdl_trigger();
  __shared__ uint8_t top[TOP_SMEM];
  const int img = blockIdx.x;
  const ImgDesc& d = B.desc[img];
  const int H = d.H, W = d.W, n = d.nlev;
  rdhei_info* info = reinterpret_cast<rdhei_info*>(d.info);

  if (owner && threadIdx.x == 0) {
    uint32_t z[10];
    const uint32_t N = (uint32_t)H * (uint32_t)W;
    for (int k = 1; k <= 8; k++) z[k] = B.hist_acc[16 * img + k - 1];
    z[0] = N; z[9] = 0;
    for (int t = 0; t <= 8; t++) info->hist[t] = t < 8 ? z[t] - z[t + 1] : z[8];
    const int lmr = d.variant == RDHEI_LMR;
    int b = d.b;
    if (b <= 0) {
      uint64_t best = 0; b = 2;
      for (int c = 2; c <= (lmr ? 8 : 7); c++) {
        uint64_t cap = (uint64_t)(lmr ? c - 1 : c) * z[c];
        if (c == 2 || cap > best) { best = cap; b = c; }
      }
    }
    info->b = b;
    info->capacity = (uint64_t)(lmr ? b - 1 : b) * z[b];
    info->status = 0;
  }

  // levels 7..n: sums of the 4 children (level 7 from the tile totals)
  for (int L = 7; L <= n; L++) {
    const int nr = H >> L, nc = W >> L;
    uint8_t* cur = top + top_off(H, W, L);
    for (int e = threadIdx.x; e < nr * nc; e += blockDim.x) {
      const int br = e / nc, bc = e % nc;
      uint32_t s = 0;
      for (int k = 0; k < 4; k++) {
        const int cr = 2 * br + (k >> 1), cc = 2 * bc + (k & 1);
        if (L == 7) s += B.sigma6[d.tile_base + (uint32_t)cr * d.tiles_x + (uint32_t)cc];
        else s += top[top_off(H, W, L - 1) + cr * (W >> (L - 1)) + cc];
      }
      cur[e] = (uint8_t)(s & 3u);
    }
    __syncthreads();
  }

  // per tile: destination under the composed rotation (bits >= 6 of the coordinates)
  const uint32_t ntiles = d.tiles_x * d.tiles_y;
  for (uint32_t t = threadIdx.x; t < ntiles; t += blockDim.x) {
    const uint32_t ty = t / d.tiles_x, tx = t % d.tiles_x;
    uint32_t a[17];
    for (int L = 0; L < 17; L++) a[L] = 0;
    for (int L = 7; L <= n; L++) {
      const uint32_t br = ty >> (L - 6), bc = tx >> (L - 6);
      if ((int)br < (H >> L) && (int)bc < (W >> L) && L >= d.lmin)
        a[L] = top[top_off(H, W, L) + br * (W >> L) + bc];
    }
    uint32_t qy = ty, qx = tx, S = 0;
    for (int j = n - 1; j >= 6; --j) {               // S_j = sum of a_L, L = j+1 .. n
      S += a[j + 1];
      const uint32_t k = j - 6;
      const uint32_t pb = (((ty >> k) & 1u) << 1) | ((tx >> k) & 1u);
      const uint32_t qb = rot_bits(ROT_FWD_LUT, S, pb);
      qy = (qy & ~(1u << k)) | ((qb >> 1) << k);
      qx = (qx & ~(1u << k)) | ((qb & 1u) << k);
    }
    const uint32_t q = qy * d.tiles_x + qx;
    if (!RDHEI_IDX_OK(B.err, q < ntiles)) continue;
    const uint8_t shi = (uint8_t)(S & 3u);           // S_6
    B.tilemap[d.tile_base + t].dec_dst = q;
    B.tilemap[d.tile_base + t].dec_shi = shi;
    B.tilemap[d.tile_base + q].enc_src = t;
    B.tilemap[d.tile_base + q].enc_shi = shi;
  }
}

// ---------------------------------------------------------------------------------
// Gather pass of the owner.  One CTA walks a run of output (rotated-domain) tiles in
// one tile row: a whole row, or 1/nsplit of it when the batch has too few rows to
// fill the GPU; per output tile Q:
//   1. source tile P = preimage of Q; P (+ left halo column) and its subtree into
//      shared memory -- fetched into registers while the previous tile was processed;
//   2. location map l (Eqs. gliding1/2 in left-neighbour form) with the chosen b;
//      EMR folds l into the pixel LSB (it becomes the LSB of I_e anyway);
//   3. rotate P into Q's frame (micro-block gather, permute.cuh);
//   4. XOR with the stashed keystream at Q (Eq. image_encryption), LMR side bits
//      into bit 7, packed rotated maps.
// ---------------------------------------------------------------------------------
template <bool ANY_LMR, bool ANY_MED>
__global__ void __launch_bounds__(256, ANY_MED ? 5 : 6) k_enc_rows(Batch B, uint32_t nsplit) {
  pdl_wait();      // the previous kernel of the operation has finished
  pdl_trigger();
  __shared__ __align__(16) uint8_t tin[TILE * TPITCH];
  __shared__ __align__(16) uint8_t tout[TILE * TPITCH];
  __shared__ __align__(16) uint8_t lin[ANY_LMR ? TILE * TPITCH : 16];
  __shared__ __align__(16) uint8_t lout[ANY_LMR ? TILE * TPITCH : 16];
  __shared__ __align__(16) uint8_t sub[SUBTREE_BYTES];
  __shared__ uint32_t selt[16];
  __shared__ uint8_t halo[TILE];
  __shared__ __align__(16) uint8_t uprow[ANY_MED ? TILE + 16 : 16];   // MED: the row above P, its left corner

  const int t = threadIdx.x;
  const uint32_t strip = blockIdx.x / nsplit, piece = blockIdx.x % nsplit;
  const int img = (int)__ldg(B.strip_owner + strip);
  const ImgDesc& d = B.desc[img];
  const int H = d.H, W = d.W;
  const rdhei_info* info = reinterpret_cast<const rdhei_info*>(d.info);
  const int b = d.b > 0 ? d.b : info->b;
  const bool LMR = ANY_LMR && d.variant == RDHEI_LMR;
  const bool med = ANY_MED && d.med != 0;
  const uint32_t tiles_x = d.tiles_x, ntiles = tiles_x * d.tiles_y;
  const uint32_t qty = strip - __ldg(B.strip_prefix + img);       // output tile row
  const uint32_t per = (tiles_x + nsplit - 1) / nsplit;
  const uint32_t tx0 = piece * per, tx1 = min(tx0 + per, tiles_x);
  if (tx0 >= tx1) return;
  const int row = t >> 2, quarter = t & 3;
  if (t < 16) selt[t] = pair_selectors(t & 3u, t >> 2);

  // source tile of output tile (qty, tx): its angle sum above level 6, my 16 bytes of
  // it, the byte left of my row (quarter 0) and one subtree word (t < 88)
  uint32_t nP = 0, nU = 0, nw[4], nhalo = 0, nsub = 0;
  uint32_t nup[4] = {0u, 0u, 0u, 0u}, ncorner = 0;              // MED: the row above the source tile
  auto fetch = [&](uint32_t tx) {
    const TileMap tm = B.tilemap[d.tile_base + qty * tiles_x + tx];
    nP = tm.enc_src;
    nU = tm.enc_shi;
    if (!RDHEI_IDX_OK(B.err, nP < ntiles)) nP = 0;
    const int py0 = (int)(nP / tiles_x) * TILE, px0 = (int)(nP % tiles_x) * TILE;
    const int y = py0 + row, x = px0 + 16 * quarter;
    int valid = (y < H) ? min(16, W - x) : 0;
    if (valid < 0) valid = 0;
    const uint8_t* sp = d.src + (size_t)y * W + x;
    if (valid == 16 && ((reinterpret_cast<uintptr_t>(sp) & 15) == 0)) {
      const uint4 v = __ldg(reinterpret_cast<const uint4*>(sp));
      nw[0] = v.x; nw[1] = v.y; nw[2] = v.z; nw[3] = v.w;
    } else {
#pragma unroll
      for (int i = 0; i < 4; i++) {
        uint32_t v = 0;
#pragma unroll
        for (int k = 0; k < 4; k++)
          if (4 * i + k < valid) v |= (uint32_t)__ldg(sp + 4 * i + k) << (8 * k);
        nw[i] = v;
      }
    }
    if (quarter == 0 && y < H) nhalo = px0 > 0 ? __ldg(d.src + (size_t)y * W + px0 - 1) : ((nw[0] & 0xFFu) ^ 0xFFu);
    if (t < SUBTREE_BYTES / 4)
      nsub = __ldg(reinterpret_cast<const uint32_t*>(B.subtree + (size_t)(d.tile_base + nP) * SUBTREE_BYTES) + t);
    if (ANY_MED && med && row == 0) {
      // the row above the tile and its upper-left corner, for the MED prediction
      const int uy = py0 - 1;
      int uv = uy >= 0 ? min(16, W - x) : 0;
      if (uv < 0) uv = 0;
      const uint8_t* up = d.src + (size_t)(uy >= 0 ? uy : 0) * W + x;
      if (uv == 16 && ((reinterpret_cast<uintptr_t>(up) & 15) == 0)) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(up));
        nup[0] = v.x; nup[1] = v.y; nup[2] = v.z; nup[3] = v.w;
      } else {
#pragma unroll
        for (int i = 0; i < 4; i++) {
          uint32_t v = 0;
#pragma unroll
          for (int k = 0; k < 4; k++)
            if (4 * i + k < uv) v |= (uint32_t)__ldg(up + 4 * i + k) << (8 * k);
          nup[i] = v;
        }
      }
      if (quarter == 0) ncorner = (uy >= 0 && px0 > 0) ? __ldg(d.src + (size_t)uy * W + px0 - 1) : 0u;
    }
  };
  fetch(tx0);

  for (uint32_t tx = tx0; tx < tx1; tx++) {
    const uint32_t P = nP, U = nU;
    const uint32_t w[4] = {nw[0], nw[1], nw[2], nw[3]};
    const int qy0 = (int)qty * TILE, qx0 = (int)tx * TILE;
    const int py0 = (int)(P / tiles_x) * TILE, px0 = (int)(P % tiles_x) * TILE;

    // 1. P, its halo column and its subtree into shared memory
    *reinterpret_cast<uint4*>(tin + row * TPITCH + 16 * quarter) = make_uint4(w[0], w[1], w[2], w[3]);
    if (quarter == 0) halo[row] = (uint8_t)nhalo;
    if (t < SUBTREE_BYTES / 4) reinterpret_cast<uint32_t*>(sub)[t] = nsub;
    if (ANY_MED && med && row == 0) {
      *reinterpret_cast<uint4*>(uprow + 16 * quarter) = make_uint4(nup[0], nup[1], nup[2], nup[3]);
      if (quarter == 0) uprow[TILE] = (uint8_t)ncorner;
    }
    if (tx + 1 < tx1) fetch(tx + 1);            // in flight while this tile is processed
    __syncthreads();

    // 2. location map with this image's b: l = 1 where the top b bits differ from the
    //    left neighbour's (first image column: always 1)
    {
      uint32_t left = quarter == 0 ? (uint32_t)halo[row] : (uint32_t)tin[row * TPITCH + 16 * quarter - 1];
      const uint32_t K = (0x80u - (0x100u >> b)) * 0x01010101u;
      uint32_t lw[4];
      if (!med) {
#pragma unroll
        for (int i = 0; i < 4; i++) {
          uint32_t prev = i == 0 ? (left << 24) : w[i - 1];
          uint32_t dd = w[i] ^ __funnelshift_l(prev, w[i], 8);
          lw[i] = ((((dd & 0x7F7F7F7Fu) + K) | dd) >> 7) & 0x01010101u;
        }
      } else {
        // related-work MED prediction from the left, upper and upper-left pixels
        const int y = py0 + row, x = px0 + 16 * quarter;
        const bool seven = d.variant == RDHEI_EMR;
        const uint8_t* ur = row > 0 ? tin + (row - 1) * TPITCH + 16 * quarter : uprow + 16 * quarter;
        uint32_t ul = quarter > 0 ? ur[-1] : row > 0 ? halo[row - 1] : uprow[TILE];
        if (px0 == 0 && quarter == 0) left = 0;
        const uint4 u4 = *reinterpret_cast<const uint4*>(ur);
        const uint32_t up[4] = {u4.x, u4.y, u4.z, u4.w};
#pragma unroll
        for (int i = 0; i < 4; i++) {
          const uint32_t A = __funnelshift_l(i == 0 ? (left << 24) : w[i - 1], w[i], 8);
          const uint32_t C = __funnelshift_l(i == 0 ? (ul << 24) : up[i - 1], up[i], 8);
          // EMR: the median of the values with the LSB cleared (twice that of the top seven bits)
          const uint32_t keep = seven ? 0xFEFEFEFEu : 0xFFFFFFFFu;
          uint32_t pred = med4(A & keep, up[i] & keep, C & keep);
          if (y == 0) pred = seven ? A & 0xFEFEFEFEu : A;                            // row 0: from the left
          if (i == 0 && x == 0) pred = (pred & 0xFFFFFF00u) | (up[0] & (seven ? 0xFEu : 0xFFu));   // column 0
          uint32_t dd = w[i] ^ pred;
          if (i == 0 && x == 0 && y == 0) dd |= 0xFFu;                               // pixel (0, 0)
          lw[i] = ((((dd & 0x7F7F7F7Fu) + K) | dd) >> 7) & 0x01010101u;
        }
      }
      __syncthreads();   // every thread has read its left byte
      if (LMR) {
        *reinterpret_cast<uint4*>(lin + row * TPITCH + 16 * quarter) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
      } else {
        *reinterpret_cast<uint4*>(tin + row * TPITCH + 16 * quarter) =
            make_uint4((w[0] & 0xFEFEFEFEu) | lw[0], (w[1] & 0xFEFEFEFEu) | lw[1],
                       (w[2] & 0xFEFEFEFEu) | lw[2], (w[3] & 0xFEFEFEFEu) | lw[3]);
      }
    }
    __syncthreads();

    // 3. rotation: output micro-block (mr, mc) <- source micro-block (pr, pc)
    {
      const uint32_t mr = t >> 4, mc = t & 15;
      uint32_t pr, pc, S1;
      enc_microblock_src(sub, U, mr, mc, pr, pc, S1);
      const uint32_t nib = sub_level1_nibbles(sub, pr, pc);
      const uint32_t sT = selt[nib & 0xF], sB = selt[nib >> 4];
      uint32_t w0, w1, w2, w3;
      ld_micro(tin, pr, pc, w0, w1, w2, w3);
      turn_subblocks(w0, w1, w2, w3, sT, sB);
      turn4x4(w0, w1, w2, w3, S1);
      st_micro(tout, mr, mc, w0, w1, w2, w3);
      if (LMR) {
        ld_micro(lin, pr, pc, w0, w1, w2, w3);
        turn_subblocks(w0, w1, w2, w3, sT, sB);
        turn4x4(w0, w1, w2, w3, S1);
        st_micro(lout, mr, mc, w0, w1, w2, w3);
      }
    }
    __syncthreads();   // also: tin, halo and sub are free for the next tile

    // 4. encrypt and store Q
    {
      const int y = qy0 + row, x = qx0 + 16 * quarter;
      int valid = (y < H) ? min(16, W - x) : 0;
      if (valid < 0) valid = 0;
      if (valid > 0) {
        const uint4 v4 = *reinterpret_cast<const uint4*>(tout + row * TPITCH + 16 * quarter);
        uint32_t v[4] = {v4.x, v4.y, v4.z, v4.w};
        const size_t off = (size_t)y * W + x;
        const uint8_t* ks = d.stash + off;
        uint8_t* dst = d.dst + off;
        const bool vec = valid == 16 && ((reinterpret_cast<uintptr_t>(ks) & 15) == 0) &&
                         ((reinterpret_cast<uintptr_t>(dst) & 15) == 0);
        uint32_t s[4];
        if (vec) {
          uint4 s4 = *reinterpret_cast<const uint4*>(ks);
          s[0] = s4.x; s[1] = s4.y; s[2] = s4.z; s[3] = s4.w;
        } else {
#pragma unroll
          for (int i = 0; i < 4; i++) {
            uint32_t a = 0;
#pragma unroll
            for (int k = 0; k < 4; k++)
              if (4 * i + k < valid) a |= (uint32_t)ks[4 * i + k] << (8 * k);
            s[i] = a;
          }
        }
        const bool plain = (W & 15) == 0;
        const uint64_t pos = (uint64_t)off;
        uint32_t e[4];
        if (!LMR) {
#pragma unroll
          for (int i = 0; i < 4; i++) e[i] = v[i] ^ (s[i] & 0xFEFEFEFEu);   // LSB = rotated l
          if (d.map_bits) put_bits16(d.map_bits, pos, flags16(v, 0), valid, plain);
        } else {
#pragma unroll
          for (int i = 0; i < 4; i++) e[i] = v[i] ^ s[i];
          if (pos < d.side_nbits && d.side_bits) {
            const uint64_t nws = (d.side_nbits + 31) >> 5;
            const uint32_t sb = stream_bits32(d.side_bits, nws, pos);    // bit c = side bit pos + c
            const int nside = (int)umin64((uint64_t)valid, d.side_nbits - pos);
#pragma unroll
            for (int i = 0; i < 4; i++) {
              const uint32_t nb = (sb >> (4 * i)) & 0xFu;
              const uint32_t spread = ((nb * 0x00204081u) & 0x01010101u) << 7;
              int nv = nside - 4 * i;
              uint32_t m = nv <= 0 ? 0u : nv >= 4 ? 0x80808080u : (0x80808080u & ((1u << (8 * nv)) - 1u));
              e[i] = (e[i] & ~m) | (spread & m);
            }
          }
          if (d.map_bits) {
            const uint4 l4 = *reinterpret_cast<const uint4*>(lout + row * TPITCH + 16 * quarter);
            const uint32_t lv[4] = {l4.x, l4.y, l4.z, l4.w};
            put_bits16(d.map_bits, pos, flags16(lv, 0), valid, plain);
          }
          if (d.eta_bits) put_bits16(d.eta_bits, pos, flags16(v, 7), valid, plain);   // Eq. MSB_map
        }
        if (vec) {
          *reinterpret_cast<uint4*>(dst) = make_uint4(e[0], e[1], e[2], e[3]);
        } else {
#pragma unroll
          for (int c = 0; c < 16; c++)
            if (c < valid) dst[c] = (uint8_t)(e[c >> 2] >> (8 * (c & 3)));
        }
      }
    }
  }
}

void launch_topmap(const Batch& B, bool owner, cudaStream_t st) {
  if (B.n_images == 0) return;
  launch_pdl(k_topmap, dim3(B.n_images), dim3(256), 0, st, B, owner ? 1 : 0);
}
void launch_enc_pass2(const Batch& B, bool any_lmr, bool any_med, cudaStream_t st) {
  if (B.total_strips == 0) return;
  // whole tile rows per CTA (the next tile's fetch hides the current one's latency),
  // split when the batch has fewer rows than ~4 CTAs per SM slot
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 1;
  const uint32_t want = (uint32_t)sms * 6u * 4u;
  uint32_t nsplit = want / B.total_strips;
  nsplit = nsplit < 1 ? 1 : nsplit > 64 ? 64 : nsplit;
  const uint32_t grid = B.total_strips * nsplit;
  if (any_med) {
    if (any_lmr) launch_pdl(k_enc_rows<true, true>, dim3(grid), dim3(256), 0, st, B, nsplit);
    else launch_pdl(k_enc_rows<false, true>, dim3(grid), dim3(256), 0, st, B, nsplit);
  } else {
    if (any_lmr) launch_pdl(k_enc_rows<true, false>, dim3(grid), dim3(256), 0, st, B, nsplit);
    else launch_pdl(k_enc_rows<false, false>, dim3(grid), dim3(256), 0, st, B, nsplit);
  }
}

}  // namespace rdhei
