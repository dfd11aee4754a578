// encode.cu -- content owner's second half: top rotation levels + choice of b
// (k_topmap) and the gather pass that labels, rotates, encrypts and embeds the map
// (k_enc_rows); and the fused owner-and-hider kernel (k_enc_fused) that goes on to
// write the K2-encrypted payload into the strip it has just encrypted.
#include "permute.cuh"
#include "slots.cuh"

namespace rdhei {

// Raw block sums (mod 4) for levels 7..n live in shared memory, row-major per level.
constexpr int TOP_SMEM = 11 * 1024;

__device__ __forceinline__ int top_off(int H, int W, int L) {
  int off = 0;
  for (int l = 7; l < L; l++) off += (H >> l) * (W >> l);
  return off;
}

constexpr int MAX_STRIPS = 1024;   // 64-row strips of the tallest image (H <= 65536)

// One CTA per image.
//   owner:    histogram -> hist[9], b (Eq. optimal_b), capacity, into rdhei_info;
//   both:     sums of the tile totals up the levels above 6 (Eq. roration) and, per
//             tile, where the composed rotation sends it and the angle sum above 6;
//   fused:    per 64-row strip of the rotated image, its payload bits (the label-0
//             pixels of its tiles times the slots per pixel) and their exclusive
//             prefix in raster order -- the bit at which the strip's slots start in the
//             concatenation of Sec. III-A-2 / III-A-3.  The owner counts its rotated
//             tiles through the tile map (a tile moves as a whole, and the in-tile
//             rotation only permutes its pixels); the receiver's tiles are already in
//             the rotated domain.  Owner: embedded = min(nbits, capacity); receiver:
//             extracted = min(max_bits, capacity), the first bit of each part when
//             the extraction splits strips (rows B.part_rows at a time, from the first
//             pass's per-tile-row counts), and the clearing of the output words that
//             two strips or parts share (and of the last, partial one): the extractor
//             writes those with atomicOr.
__global__ void __launch_bounds__(256) k_topmap(Batch B, int owner, int fused) {
  pdl_wait();      // the previous kernel of the operation has finished
  pdl_trigger();
  __shared__ uint8_t top[TOP_SMEM];
  __shared__ uint32_t strip_acc[MAX_STRIPS];
  __shared__ int s_b;
  const int img = blockIdx.x;
  const ImgDesc& d = B.desc[img];
  const int H = d.H, W = d.W, n = d.nlev;
  rdhei_info* info = reinterpret_cast<rdhei_info*>(d.info);
  const int lmr = d.variant == RDHEI_LMR;

  if (threadIdx.x == 0) {
    if (owner) {
      uint32_t z[10];
      const uint32_t N = (uint32_t)H * (uint32_t)W;
      for (int k = 1; k <= 8; k++) z[k] = B.hist_acc[16 * img + k - 1];
      z[0] = N; z[9] = 0;
      for (int t = 0; t <= 8; t++) info->hist[t] = t < 8 ? z[t] - z[t + 1] : z[8];
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
      s_b = b;
    } else {
      s_b = d.b > 0 ? d.b : info->b;
    }
  }
  if (fused)
    for (uint32_t i = threadIdx.x; i < d.tiles_y; i += blockDim.x) strip_acc[i] = 0u;
  __syncthreads();
  const int b = s_b;

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
    if (fused) {
      // label-0 pixels of the rotated tile: the owner's source tile t lands on q, the
      // receiver's tile t is already a rotated one
      const uint32_t cnt = B.tile_cnt[8 * (size_t)(d.tile_base + t) + (owner ? b - 1 : 0)];
      atomicAdd(&strip_acc[owner ? qy : ty], cnt);
    }
    if (!RDHEI_IDX_OK(B.err, q < ntiles)) continue;
    const uint8_t shi = (uint8_t)(S & 3u);           // S_6
    B.tilemap[d.tile_base + t].dec_dst = q;
    B.tilemap[d.tile_base + t].dec_shi = shi;
    B.tilemap[d.tile_base + q].enc_src = t;
    B.tilemap[d.tile_base + q].enc_shi = shi;
  }
  if (!fused) return;
  __syncthreads();

  // strips: payload bits and their exclusive prefix (one warp; <= 1024 strips, 32 per lane)
  const uint32_t slots = (uint32_t)(lmr ? b - 1 : b);
  const uint32_t ns = d.tiles_y, sbase = __ldg(B.strip_prefix + img);
  if (threadIdx.x < 32) {
    const uint32_t lane = threadIdx.x, per = (ns + 31) / 32;
    const uint32_t i0 = lane * per, i1 = min(i0 + per, ns);
    uint32_t sum = 0;
    for (uint32_t i = i0; i < i1; i++) sum += strip_acc[i] * slots;
    uint32_t inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xffffffffu, inc, o);
      if ((int)lane >= o) inc += u;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, inc, 31);
    uint32_t run = inc - sum;
    for (uint32_t i = i0; i < i1; i++) {
      const uint32_t v = strip_acc[i] * slots;
      B.strip_base[sbase + i] = run;
      B.strip_tot[sbase + i] = v;
      run += v;
    }
    if (lane == 0) {
      if (owner) {
        info->embedded = umin64(d.nbits, total);
        if (d.nbits > total) { info->status = ERR_CAPACITY; set_error(B.err, ERR_CAPACITY); }
      } else {
        info->extracted = umin64(d.max_bits, total);
      }
    }
  }
  if (owner) return;
  __syncthreads();
  const uint64_t E = info->extracted;
  uint32_t* out = reinterpret_cast<uint32_t*>(d.bits_out);
  const int R = B.part_rows, parts = TILE / R;
  if (parts > 1) {
    // slots of each part (R rows of a strip), one warp per part: lanes take the strip's
    // tiles, four row counts per 32-bit load (rows below the image count 0)
    const uint32_t tiles_x = d.tiles_x, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (uint32_t e = threadIdx.x >> 5; e < ns * (uint32_t)parts; e += nwarps) {
      const uint32_t st = e / parts, k = e - st * parts;
      const uint32_t* rc = reinterpret_cast<const uint32_t*>(
          B.rowcnt + ((size_t)d.tile_base + (size_t)st * tiles_x) * TILE + (size_t)k * R);
      uint32_t c = 0;
      for (uint32_t tx = lane; tx < tiles_x; tx += 32)
        for (int q = 0; q < R / 4; q++) c = __dp4a(rc[(size_t)tx * (TILE / 4) + q], 0x01010101u, c);
      c = __reduce_add_sync(0xffffffffu, c);
      if (lane == 0) B.part_base[(size_t)(sbase + st) * MAX_PARTS + k] = c * slots;
    }
    __syncthreads();
    // within each strip: exclusive prefix from the strip's first bit; a part boundary
    // inside a word clears that word
    for (uint32_t st = threadIdx.x; st < ns; st += blockDim.x) {
      uint32_t* pb = B.part_base + (size_t)(sbase + st) * MAX_PARTS;
      uint64_t run = B.strip_base[sbase + st];
      for (int k = 0; k < parts; k++) {
        const uint32_t v = pb[k];
        pb[k] = (uint32_t)run;
        if (k > 0 && run < E && (run & 31u)) out[run >> 5] = 0u;
        run += v;
      }
    }
  }
  // the words two strips share, and the last partial word
  for (uint32_t st = threadIdx.x + 1; st < ns; st += blockDim.x) {
    const uint64_t G = B.strip_base[sbase + st];
    if (G < E && (G & 31u)) out[G >> 5] = 0u;
  }
  if (threadIdx.x == 0 && (E & 31u)) out[E >> 5] = 0u;
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
struct EncSmem {
  __align__(16) uint8_t tin[TILE * TPITCH];
  __align__(16) uint8_t tout[TILE * TPITCH];
  __align__(16) uint8_t lin[ANY_LMR ? TILE * TPITCH : 16];
  __align__(16) uint8_t lout[ANY_LMR ? TILE * TPITCH : 16];
  __align__(16) uint8_t sub[SUBTREE_BYTES];
  uint32_t selt[16];
  uint8_t halo[TILE];
  __align__(16) uint8_t uprow[ANY_MED ? TILE + 16 : 16];   // MED: the row above P, its left corner
};

// Output tiles [tx0, tx1) of one output tile row (`piece` of `nsplit` pieces).  `pre`
// runs once, while the loads of the first source tile are in flight.
struct NoPre {
  __device__ __forceinline__ void operator()() const {}
};
// SKEW: the source tile and label plane in the chunk-skewed layout (skewed_chunk).
template <bool ANY_LMR, bool ANY_MED, bool SKEW = false, typename Pre = NoPre>
__device__ __forceinline__ void enc_rows_body(const Batch& B, uint32_t strip, uint32_t nsplit, uint32_t piece,
                                              EncSmem<ANY_LMR, ANY_MED>& sm, const Pre& pre = Pre()) {
  uint8_t* const tin = sm.tin;
  uint8_t* const tout = sm.tout;
  uint8_t* const lin = sm.lin;
  uint8_t* const lout = sm.lout;
  uint8_t* const sub = sm.sub;
  uint32_t* const selt = sm.selt;
  uint8_t* const halo = sm.halo;
  uint8_t* const uprow = sm.uprow;

  const int t = threadIdx.x;
  const int img = (int)__ldg(B.strip_owner + strip);
  const ImgDesc& d = B.desc[img];
  const int H = d.H, W = d.W;
  const rdhei_info* info = reinterpret_cast<const rdhei_info*>(d.info);
  const int b = d.b > 0 ? d.b : info->b;
  const bool LMR = ANY_LMR && d.variant == RDHEI_LMR;
  const bool med = ANY_MED && d.med != 0;
  const uint32_t tiles_x = d.tiles_x, ntiles = tiles_x * d.tiles_y;
  (void)ntiles;                                                  // index checks only
  const uint32_t qty = strip - __ldg(B.strip_prefix + img);       // output tile row
  const uint32_t per = (tiles_x + nsplit - 1) / nsplit;
  const uint32_t tx0 = piece * per, tx1 = min(tx0 + per, tiles_x);
  if (tx0 >= tx1) return;
  const int row = tile_row_of(t), quarter = t & 3;
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
  pre();

  for (uint32_t tx = tx0; tx < tx1; tx++) {
    const uint32_t P = nP, U = nU;
    const uint32_t w[4] = {nw[0], nw[1], nw[2], nw[3]};
    const int qy0 = (int)qty * TILE, qx0 = (int)tx * TILE;
    const int py0 = (int)(P / tiles_x) * TILE, px0 = (int)(P % tiles_x) * TILE;

    // 1. P, its halo column and its subtree into shared memory
    *reinterpret_cast<uint4*>(skewed_chunk<SKEW>(tin, row, quarter)) = make_uint4(w[0], w[1], w[2], w[3]);
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
      uint32_t left = quarter == 0 ? (uint32_t)halo[row] : (uint32_t)skewed_chunk<SKEW>(tin, row, quarter - 1)[15];
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
        const uint8_t* ur = row > 0 ? skewed_chunk<SKEW>(tin, row - 1, quarter) : uprow + 16 * quarter;
        uint32_t ul = quarter > 0 ? (row > 0 ? skewed_chunk<SKEW>(tin, row - 1, quarter - 1)[15] : ur[-1])
                                  : row > 0 ? halo[row - 1] : uprow[TILE];
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
        *reinterpret_cast<uint4*>(skewed_chunk<SKEW>(lin, row, quarter)) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
      } else {
        *reinterpret_cast<uint4*>(skewed_chunk<SKEW>(tin, row, quarter)) =
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
      ld_micro_skewed<SKEW>(tin, pr, pc, w0, w1, w2, w3);
      turn_subblocks(w0, w1, w2, w3, sT, sB);
      turn4x4(w0, w1, w2, w3, S1);
      st_micro(tout, mr, mc, w0, w1, w2, w3);
      if (LMR) {
        ld_micro_skewed<SKEW>(lin, pr, pc, w0, w1, w2, w3);
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
        const uint32_t pos = (uint32_t)off;                         // < 2^27: 32-bit stream positions
        uint32_t e[4];
        if (!LMR) {
#pragma unroll
          for (int i = 0; i < 4; i++) e[i] = v[i] ^ (s[i] & 0xFEFEFEFEu);   // LSB = rotated l
          if (d.map_bits) put_bits16(d.map_bits, pos, flags16(v, 0), valid, plain);
        } else {
#pragma unroll
          for (int i = 0; i < 4; i++) e[i] = v[i] ^ s[i];
          if (pos < d.side_nbits && d.side_bits) {
            const uint32_t nws = (uint32_t)((d.side_nbits + 31) >> 5);
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

template <bool ANY_LMR, bool ANY_MED>
__global__ void __launch_bounds__(256, ANY_MED ? 5 : 6) k_enc_rows(Batch B, uint32_t nsplit) {
  pdl_wait();      // the previous kernel of the operation has finished
  pdl_trigger();
  __shared__ EncSmem<ANY_LMR, ANY_MED> sm;
  enc_rows_body<ANY_LMR, ANY_MED>(B, blockIdx.x / nsplit, nsplit, blockIdx.x % nsplit, sm);
}

// Hider's half of the fused encode (Sec. III-A-2 / III-B-2) for one 64-row strip of
// the rotated image that this CTA has just encrypted: its slots start at stream bit
// strip_base (k_topmap), so the 8192-pixel chunks are walked in raster order with a
// running offset.  The message words are K2-encrypted (e = m XOR z2) into a window of
// shared memory, one ChaCha20 block per thread: the strip's first window while the
// gather's first loads are in flight, the next one whenever a chunk's slots run past
// it (wide strips).  Per chunk: the strip's pixels come back from L2 (written moments
// ago by this CTA; the next chunk is not prefetched: its registers would cost the
// fifth resident CTA per SM), a block scan places each thread's slots and spread_slots
// writes them.
constexpr int WINDOW_WORDS = 16 * 255;   // message words staged at once: at most 256 ChaCha20 blocks
struct EmbedSmem {
  uint32_t ebuf[WINDOW_WORDS + 1];
  uint32_t warp_tot[HIDE_THREADS / 32];
  SlotTables tabs;
};

// e words [w_lo, w_lo + nw) of image d's message into buf (MSB-first), and a zero word
// after them; one ChaCha20 block of z2 per thread (nw <= WINDOW_WORDS: <= 256 blocks)
__device__ __forceinline__ void stage_message(const ImgDesc& d, uint64_t w_lo, uint32_t nw, uint32_t* buf) {
  const int t = threadIdx.x;
  const uint64_t j0 = w_lo >> 4;
  const uint32_t nblk = (uint32_t)(((w_lo + nw - 1) >> 4) - j0 + 1);
  const uint32_t* pay = reinterpret_cast<const uint32_t*>(d.payload);
  if ((uint32_t)t < nblk) {
    uint32_t o[16];
    const uint64_t j = j0 + t;
    chacha20_block<2>(d.k2, (uint32_t)j, d.n2, o, d.one);
    // word i of the block is window word 16 t + i - o0, o0 = w_lo's offset in block j0
    const uint32_t o0 = (uint32_t)(w_lo & 15);
    const uint32_t* pj = pay + 16 * j;
#pragma unroll
    for (int i = 0; i < 16; i++) {
      const uint32_t k = 16u * (uint32_t)t + (uint32_t)i - o0;      // wraps (large) before the window
      if (k < nw) buf[k] = bswap32(__ldg(pj + i) ^ o[i]);
    }
  }
  if (t == 0) buf[nw] = 0u;
}

struct StripRange {
  uint64_t G0, send;
};
__device__ __forceinline__ StripRange strip_range(const Batch& B, uint32_t s, const ImgDesc& d) {
  const rdhei_info* info = reinterpret_cast<const rdhei_info*>(d.info);
  const uint64_t G0 = B.strip_base[s];
  return {G0, umin64(G0 + B.strip_tot[s], info->embedded)};
}

// the window of message words that starts at stream word w0: up to WINDOW_WORDS, not
// past the strip's last slot
__device__ __forceinline__ uint32_t window_words(uint64_t w0, uint64_t send) {
  return (uint32_t)umin64(WINDOW_WORDS, ((send - 1) >> 5) - w0 + 1);
}

// the strip's first window (called while phase 1's loads fly)
__device__ __forceinline__ void stage_strip(const Batch& B, uint32_t s, EmbedSmem& sm) {
  const ImgDesc& d = B.desc[__ldg(B.strip_owner + s)];
  const StripRange r = strip_range(B, s, d);
  if (r.send > r.G0) stage_message(d, r.G0 >> 5, window_words(r.G0 >> 5, r.send), sm.ebuf);
}

__device__ __forceinline__ void embed_strip(const Batch& B, uint32_t s, EmbedSmem& sm) {
  const int t = threadIdx.x;
  init_slot_tables(sm.tabs);
  const int img = (int)__ldg(B.strip_owner + s);
  const ImgDesc& d = B.desc[img];
  const rdhei_info* info = reinterpret_cast<const rdhei_info*>(d.info);
  const uint32_t ty = s - __ldg(B.strip_prefix + img);
  const uint64_t W = (uint64_t)d.W;
  const uint64_t p0 = (uint64_t)ty * TILE * W, p1 = (uint64_t)min((int)(ty + 1) * TILE, d.H) * W;
  const StripRange r = strip_range(B, s, d);
  __syncthreads();   // tables; the first window (written before phase 1's first barrier)
  if (r.G0 >= r.send) return;
  const uint64_t Wb = r.G0 >> 5;                             // the first staged window: words [Wb, Wb + Wn)
  uint32_t Wn = window_words(Wb, r.send);
  const uint32_t slots = (uint32_t)slots_of(d, info);
  const uint32_t fshift = (d.variant == RDHEI_LMR ? 7u : 8u) - slots;
  // 32-bit positions: pixels from the strip's first, stream bits from B0, the start of
  // the first window's first word (the strip holds < 2^22 pixels of <= 7 slot bits)
  const uint64_t B0 = 32 * Wb;
  uint8_t* const sdst = d.dst + p0;
  const uint32_t npx = (uint32_t)(p1 - p0), send = (uint32_t)(r.send - B0);
  uint32_t wb = 0;                                           // the window's first word, relative to Wb
  uint32_t g = (uint32_t)(r.G0 - B0);
  for (uint32_t c0 = 0; c0 < npx && g < send; c0 += SCAN_PX) {
    ChunkPx cur;
    const uint32_t q0 = c0 + (uint32_t)HIDE_PX * t;
    load_strip_run(d, sdst, p0, q0, npx, cur);
    const uint32_t zmask = zero_mask(d, cur);
    uint32_t Tc;
    const uint32_t my_off = block_exclusive_scan((uint32_t)__popc(zmask) * slots, sm.warp_tot, Tc);
    const uint32_t endc = min(g + Tc, send);
    if (endc > g) {
      const uint32_t w_lo = g >> 5;
      if (((endc - 1) >> 5) >= wb + Wn) {
        // the chunk's slots run past the window: the next window starts at its first word
        // (the block scan's barriers ordered every earlier read of the buffer)
        wb = w_lo;
        Wn = window_words(Wb + wb, r.send);
        stage_message(d, Wb + wb, Wn, sm.ebuf);
        __syncthreads();
      }
      const uint32_t k0 = g + my_off;
      if (zmask && k0 < endc) {
        spread_slots(cur.px, zmask, slots, fshift, sm.ebuf + (w_lo - wb), 32 * w_lo, k0, endc, sm.tabs, B.err);
        uint8_t* dst = sdst + q0;
        if (cur.valid == HIDE_PX && ((reinterpret_cast<uintptr_t>(dst) & 15) == 0)) {
          __stcg(reinterpret_cast<uint4*>(dst), make_uint4(cur.px[0], cur.px[1], cur.px[2], cur.px[3]));
          __stcg(reinterpret_cast<uint4*>(dst) + 1, make_uint4(cur.px[4], cur.px[5], cur.px[6], cur.px[7]));
        } else {
#pragma unroll
          for (int k = 0; k < HIDE_PX; k++)
            if (k < cur.valid) dst[k] = (uint8_t)(cur.px[k >> 2] >> (8 * (k & 3)));
        }
      }
    }
    g += Tc;
  }
}

// Fused owner + hider (Sec. III-A-1 then III-A-2; III-B-1 then III-B-2): one CTA per
// 64-row strip of the rotated image gathers, labels, rotates and encrypts its tiles
// (as k_enc_rows) and then embeds the payload into that strip.  Five CTAs per SM
// (48 registers) measured faster than four (64) or six (40, more spills).
template <bool ANY_LMR, bool ANY_MED>
__global__ void __launch_bounds__(256, 5) k_enc_fused(Batch B) {
  pdl_wait();      // the previous kernel of the operation has finished
  pdl_trigger();
  __shared__ EncSmem<ANY_LMR, ANY_MED> sm;
  __shared__ EmbedSmem em;
  const uint32_t s = blockIdx.x;
  enc_rows_body<ANY_LMR, ANY_MED, true>(B, s, 1, 0, sm, [&]() { stage_strip(B, s, em); });
  __syncthreads();   // the strip's encrypted pixels (and LMR map bits) are in global memory
  embed_strip(B, s, em);
}

void launch_topmap(const Batch& B, bool owner, bool fused, cudaStream_t st) {
  if (B.n_images == 0) return;
  launch_pdl(k_topmap, dim3(B.n_images), dim3(256), 0, st, B, owner ? 1 : 0, fused ? 1 : 0);
}
void launch_enc_fused(const Batch& B, bool any_lmr, bool any_med, cudaStream_t st) {
  if (B.total_strips == 0) return;
  const dim3 grid(B.total_strips), block(256);
  if (any_med) {
    if (any_lmr) launch_pdl(k_enc_fused<true, true>, grid, block, 0, st, B);
    else launch_pdl(k_enc_fused<false, true>, grid, block, 0, st, B);
  } else {
    if (any_lmr) launch_pdl(k_enc_fused<true, false>, grid, block, 0, st, B);
    else launch_pdl(k_enc_fused<false, false>, grid, block, 0, st, B);
  }
}
void launch_enc_pass2(const Batch& B, bool any_lmr, bool any_med, uint32_t nsplit, cudaStream_t st) {
  if (B.total_strips == 0) return;
  // whole tile rows per CTA (the next tile's fetch hides the current one's latency),
  // split when the batch has fewer rows than ~4 CTAs per SM slot (unless the plan fixes
  // the split)
  if (nsplit == 0) {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 1;
    const uint32_t want = (uint32_t)sms * 6u * 4u;
    nsplit = want / B.total_strips;
    nsplit = nsplit < 1 ? 1 : nsplit > 64 ? 64 : nsplit;
  }
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
