// api.cu -- host side of the C ABI (include/rdhei.h): validation, workspace layout,
// descriptor upload and kernel launch order.  No device memory is allocated here.
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/rdhei.h"
#include "common.cuh"

namespace rdhei {
void launch_pass1(const Batch& B, int mode, bool general, bool any_med, cudaStream_t st);
void launch_topmap(const Batch& B, bool owner, bool fused, cudaStream_t st);
void launch_enc_fused(const Batch& B, bool any_lmr, bool any_med, cudaStream_t st);
void launch_extract_strips(const Batch& B, cudaStream_t st);
void launch_enc_pass2(const Batch& B, bool any_lmr, bool any_med, uint32_t nsplit, cudaStream_t st);
cudaError_t launch_zero(void* p, size_t bytes, cudaStream_t st);
void launch_dec_pass2(const Batch& B, bool any_lmr, bool any_med, cudaStream_t st);
void launch_count(const Batch& B, bool extract, cudaStream_t st);
void launch_offsets(const Batch& B, bool extract, cudaStream_t st);
void launch_z2_count(const Batch& B, cudaStream_t st);
void launch_scan(const Batch& B, bool extract, cudaStream_t st);
void launch_z2_xor(const Batch& B, bool decrypt, cudaStream_t st);
void launch_lmr_side(const Batch& B, cudaStream_t st);
void launch_med_wave(const Batch& B, cudaStream_t st);
}  // namespace rdhei

using namespace rdhei;

struct rdhei_plan {
  std::vector<rdhei_job> jobs;
  std::vector<ImgDesc> desc;
  std::vector<uint32_t> tile_prefix, chunk_prefix, z2_prefix, strip_prefix;
  std::vector<uint2> wave_list;          // MED recovery tiles in anti-diagonal order
  std::vector<uint32_t> tile_owner, strip_owner;   // image of each global tile / strip
  std::vector<size_t> stash_off, ebuf_off;
  size_t off_err = 0, off_zero = 0, zero_bytes = 0, off_tickets = 0, off_hist = 0, off_chunk_status = 0,
         off_tile_flags = 0, off_desc = 0, off_tile_prefix = 0, off_chunk_prefix = 0, off_z2_prefix = 0, off_strip_prefix = 0, off_tile_rows = 0,
         off_subtree = 0, off_aux = 0, off_sigma6 = 0, off_tilemap = 0, off_wave_flags = 0, off_wave_list = 0,
         off_lab = 0, off_tile_owner = 0, off_strip_owner = 0, off_tile_cnt = 0, off_strip_base = 0,
         off_strip_tot = 0, off_rowcnt = 0, off_part_base = 0, total = 0;
  uint32_t total_tiles = 0, total_chunks = 0, total_z2 = 0, total_strips = 0, total_wave = 0;
  int wave_cols = WAVE_COLS_DEFAULT;
  int extract_rows = 0;                  // rows per k_extract_strips CTA (0 = chosen per batch)
  int auto_rows = 0;                     // the choice for 0, made once
  int enc_split = 0;                     // k_enc_rows CTAs per tile row (0 = chosen per batch)
  bool any_lmr = false, general = false, any_med = false;
  void* ws = nullptr;
  Batch batch{};
};

static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

static int levels_of(int H, int W) {
  int m = H < W ? H : W, n = 0;
  while ((2 << n) <= m) n++;
  return n;
}

static int validate_job(const rdhei_job& j) {
  if (j.H < 1 || j.W < 1 || j.H > 65536 || j.W > 65536) return RDHEI_EINVAL;
  if ((uint64_t)j.H * (uint64_t)j.W > (1ull << 27)) return RDHEI_EINVAL;
  if (j.variant < RDHEI_EMR || j.variant > RDHEI_LMR_MED) return RDHEI_EINVAL;
  const int bmax = (j.variant & 1) == RDHEI_EMR ? 7 : 8;
  if (j.b != 0 && (j.b < 2 || j.b > bmax)) return RDHEI_EINVAL;
  if (j.rot_lmin < 0 || j.rot_lmin > 16) return RDHEI_EINVAL;
  if (!j.info) return RDHEI_EINVAL;
  if (reinterpret_cast<uintptr_t>(j.info) & 7) return RDHEI_EINVAL;
  return RDHEI_OK;
}

// MED recovery work list.  Tile mode (wave_cols 64 / 128 / 256): tiles of 32 x wave_cols,
// ordered by anti-diagonal (ty + tx) across all images, so every tile's upper and left
// neighbours come earlier in the list.  Band mode (wave_cols 0): one entry per MED image.
static int layout_wave(rdhei_plan* p) {
  const int n = (int)p->jobs.size();
  if (p->wave_cols == 0) {
    p->wave_list.clear();
    for (int i = 0; i < n; i++)
      if (p->desc[i].med) p->wave_list.push_back(make_uint2((uint32_t)i, 0u));
    p->total_wave = (uint32_t)p->wave_list.size();
    return RDHEI_OK;
  }
  const uint32_t wc = (uint32_t)p->wave_cols;
  uint32_t maxdiag = 0;
  uint64_t wave = 0;
  for (int i = 0; i < n; i++) {
    ImgDesc& d = p->desc[i];
    if (!d.med) continue;
    const uint32_t wty = (uint32_t)((d.H + WAVE_ROWS - 1) / WAVE_ROWS);
    d.wave_tx = (uint32_t)((d.W + wc - 1) / wc);
    d.wave_base = (uint32_t)wave;
    wave += (uint64_t)wty * d.wave_tx;
    if (wty + d.wave_tx - 1 > maxdiag) maxdiag = wty + d.wave_tx - 1;
  }
  if (wave >= (1ull << 31)) return RDHEI_EINVAL;
  p->total_wave = (uint32_t)wave;
  p->wave_list.clear();
  p->wave_list.reserve(wave);
  for (uint32_t dg = 0; dg < maxdiag; dg++)
    for (int i = 0; i < n; i++) {
      const ImgDesc& d = p->desc[i];
      if (!d.med) continue;
      const uint32_t wty = (uint32_t)((d.H + WAVE_ROWS - 1) / WAVE_ROWS);
      for (uint32_t ty = 0; ty < wty && ty <= dg; ty++) {
        const uint32_t tx = dg - ty;
        if (tx < d.wave_tx) p->wave_list.push_back(make_uint2((uint32_t)i, (ty << 16) | tx));
      }
    }
  return RDHEI_OK;
}

static void build_layout(rdhei_plan* p) {
  const int n = (int)p->jobs.size();
  size_t off = 0;
  p->off_err = off;                      // zero region starts with the error word
  p->off_zero = off;
  p->off_tickets = off + 16;
  off = align_up(off + 16 + 8 * 4, 256);
  p->off_hist = off;
  off = align_up(off + (size_t)n * 16 * 4, 256);
  p->off_chunk_status = off;
  off = align_up(off + (size_t)p->total_chunks * 8, 256);
  p->off_tile_flags = off;
  off = align_up(off + (size_t)p->total_tiles * 4, 256);
  p->off_wave_flags = off;
  off = align_up(off + (size_t)p->total_wave * 4, 256);
  p->zero_bytes = off - p->off_zero;
  p->off_desc = off;
  off = align_up(off + (size_t)n * sizeof(ImgDesc), 256);
  p->off_tile_prefix = off;
  off = align_up(off + (size_t)(n + 1) * 4, 256);
  p->off_chunk_prefix = off;
  off = align_up(off + (size_t)(n + 1) * 4, 256);
  p->off_z2_prefix = off;
  off = align_up(off + (size_t)(n + 1) * 4, 256);
  p->off_strip_prefix = off;
  off = align_up(off + (size_t)(n + 1) * 4, 256);
  p->off_wave_list = off;
  off = align_up(off + (size_t)p->total_wave * sizeof(uint2), 256);
  p->off_tile_owner = off;
  off = align_up(off + (size_t)p->total_tiles * 4, 256);
  p->off_strip_owner = off;
  off = align_up(off + (size_t)p->total_strips * 4, 256);
  p->off_tile_rows = off;
  off = align_up(off + (size_t)p->total_tiles * 128, 256);
  p->off_subtree = off;
  off = align_up(off + (size_t)p->total_tiles * SUBTREE_BYTES, 256);
  p->off_aux = off;
  off = align_up(off + (size_t)p->total_tiles * AUX_BYTES, 256);
  p->off_sigma6 = off;
  off = align_up(off + (size_t)p->total_tiles, 256);
  p->off_tilemap = off;
  off = align_up(off + (size_t)p->total_tiles * sizeof(TileMap), 256);
  p->off_lab = off;
  if (p->any_med) off = align_up(off + (size_t)p->total_tiles * AUX_BYTES, 256);
  p->off_tile_cnt = off;
  off = align_up(off + (size_t)p->total_tiles * 16, 256);
  p->off_strip_base = off;
  off = align_up(off + (size_t)p->total_strips * 4, 256);
  p->off_strip_tot = off;
  off = align_up(off + (size_t)p->total_strips * 4, 256);
  p->off_rowcnt = off;
  off = align_up(off + (size_t)p->total_tiles * TILE, 256);
  p->off_part_base = off;
  off = align_up(off + (size_t)p->total_strips * MAX_PARTS * 4, 256);
  p->stash_off.resize(n);
  p->ebuf_off.resize(n);
  for (int i = 0; i < n; i++) {
    p->stash_off[i] = off;
    off = align_up(off + (size_t)p->jobs[i].H * p->jobs[i].W, 256);
    p->ebuf_off[i] = off;
    off = align_up(off + (size_t)((p->jobs[i].nbits + 31) / 32) * 4, 256);
  }
  p->total = off;
}

extern "C" {

int rdhei_plan_create(const rdhei_job* jobs, int n, rdhei_plan** out) {
  if (!out || n < 0 || (n > 0 && !jobs)) return RDHEI_EINVAL;
  *out = nullptr;
  rdhei_plan* p = new (std::nothrow) rdhei_plan();
  if (!p) return RDHEI_EINVAL;
  p->jobs.assign(jobs, jobs + n);
  p->desc.resize(n);
  p->tile_prefix.resize(n + 1);
  p->chunk_prefix.resize(n + 1);
  p->z2_prefix.resize(n + 1);
  p->strip_prefix.resize(n + 1);
  uint64_t tiles = 0, chunks = 0, z2 = 0, strips = 0;
  for (int i = 0; i < n; i++) {
    const rdhei_job& j = p->jobs[i];
    int rc = validate_job(j);
    if (rc) { delete p; return rc; }
    ImgDesc& d = p->desc[i];
    std::memset(&d, 0, sizeof(d));
    d.H = j.H; d.W = j.W; d.variant = j.variant & 1; d.b = j.b;
    d.med = j.variant >> 1;
    d.one = 1;
    d.nlev = levels_of(j.H, j.W);
    int lmin = j.rot_lmin > 0 ? j.rot_lmin : (d.variant == RDHEI_EMR ? 1 : 4);
    if (d.nlev >= 1 && lmin > d.nlev) lmin = d.nlev;
    d.lmin = j.rot_enable ? lmin : NO_ROTATION;
    d.tiles_x = (uint32_t)((j.W + TILE - 1) / TILE);
    d.tiles_y = (uint32_t)((j.H + TILE - 1) / TILE);
    d.nchunks = (uint32_t)(((uint64_t)j.H * j.W + CHUNK_PX - 1) / CHUNK_PX);
    d.tile_base = (uint32_t)tiles;
    d.chunk_base = (uint32_t)chunks;
    p->tile_prefix[i] = (uint32_t)tiles;
    p->chunk_prefix[i] = (uint32_t)chunks;
    p->z2_prefix[i] = (uint32_t)z2;
    p->strip_prefix[i] = (uint32_t)strips;
    strips += d.tiles_y;
    tiles += (uint64_t)d.tiles_x * d.tiles_y;
    chunks += d.nchunks;
    // K2 keystream blocks (512 message bits each) for the hider's or receiver's message
    const uint64_t capped = j.max_bits < 7ull * j.H * j.W ? j.max_bits : 7ull * j.H * j.W;
    const uint64_t mbits = j.nbits > capped ? j.nbits : capped;
    z2 += (mbits + 511) / 512;
    for (int k = 0; k < 8; k++) {
      d.k1[k] = (uint32_t)j.k1[4 * k] | ((uint32_t)j.k1[4 * k + 1] << 8) | ((uint32_t)j.k1[4 * k + 2] << 16) |
                ((uint32_t)j.k1[4 * k + 3] << 24);
      d.k2[k] = (uint32_t)j.k2[4 * k] | ((uint32_t)j.k2[4 * k + 1] << 8) | ((uint32_t)j.k2[4 * k + 2] << 16) |
                ((uint32_t)j.k2[4 * k + 3] << 24);
    }
    for (int k = 0; k < 3; k++) {
      d.n1[k] = (uint32_t)j.nonce1[4 * k] | ((uint32_t)j.nonce1[4 * k + 1] << 8) |
                ((uint32_t)j.nonce1[4 * k + 2] << 16) | ((uint32_t)j.nonce1[4 * k + 3] << 24);
      d.n2[k] = (uint32_t)j.nonce2[4 * k] | ((uint32_t)j.nonce2[4 * k + 1] << 8) |
                ((uint32_t)j.nonce2[4 * k + 2] << 16) | ((uint32_t)j.nonce2[4 * k + 3] << 24);
    }
    d.src = j.src; d.dst = j.dst; d.map_bits = j.map_bits; d.eta_bits = j.eta_bits;
    d.side_bits = j.side_bits; d.side_nbits = j.side_nbits;
    d.payload = j.payload; d.nbits = j.nbits;
    d.bits_out = j.bits_out;
    // no image holds more than 7 bits per pixel: larger requests are capped there
    d.max_bits = j.max_bits < 7ull * j.H * j.W ? j.max_bits : 7ull * j.H * j.W;
    d.info = j.info;
    if (d.variant == RDHEI_LMR) p->any_lmr = true;
    if (d.med) p->any_med = true;
    if (j.W % 64) p->general = true;
  }
  if (layout_wave(p) != RDHEI_OK) { delete p; return RDHEI_EINVAL; }
  if (tiles >= (1ull << 32) || chunks >= (1ull << 32) || z2 >= (1ull << 32)) { delete p; return RDHEI_EINVAL; }
  p->tile_prefix[n] = (uint32_t)tiles;
  p->chunk_prefix[n] = (uint32_t)chunks;
  p->z2_prefix[n] = (uint32_t)z2;
  p->strip_prefix[n] = (uint32_t)strips;
  p->total_strips = (uint32_t)strips;
  p->total_z2 = (uint32_t)z2;
  p->total_tiles = (uint32_t)tiles;
  p->total_chunks = (uint32_t)chunks;
  p->tile_owner.resize(p->total_tiles);
  p->strip_owner.resize(p->total_strips);
  for (int i = 0; i < n; i++) {
    for (uint32_t t = p->tile_prefix[i]; t < p->tile_prefix[i + 1]; t++) p->tile_owner[t] = (uint32_t)i;
    for (uint32_t t = p->strip_prefix[i]; t < p->strip_prefix[i + 1]; t++) p->strip_owner[t] = (uint32_t)i;
  }
  build_layout(p);
  *out = p;
  return RDHEI_OK;
}

size_t rdhei_plan_workspace_size(const rdhei_plan* p) { return p ? p->total : 0; }

size_t rdhei_plan_staging_size(const rdhei_plan* p) {
  return p ? p->off_strip_owner + (size_t)p->total_strips * 4 - p->off_desc : 0;
}

// Descriptors, prefixes and owner tables as one host image of the workspace's
// descriptor region, copied once: from `staging` (caller-owned, page-locked, valid until
// the stream passes the copy) without waiting, else from a temporary host buffer and
// waiting for the copy.
static int upload_impl(rdhei_plan* p, void* ws, size_t ws_bytes, void* staging, size_t staging_bytes,
                       void* stream) {
  if (!p || !ws) return RDHEI_EINVAL;
  if (ws_bytes < p->total) return RDHEI_ESPACE;
  if (reinterpret_cast<uintptr_t>(ws) & 255) return RDHEI_EINVAL;
  const size_t lo = p->off_desc, hi = p->off_strip_owner + (size_t)p->total_strips * 4;
  if (staging && staging_bytes < hi - lo) return RDHEI_ESPACE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  uint8_t* base = reinterpret_cast<uint8_t*>(ws);
  const int n = (int)p->jobs.size();
  for (int i = 0; i < n; i++) {
    p->desc[i].stash = base + p->stash_off[i];
    p->desc[i].ebuf = base + p->ebuf_off[i];
  }
  std::vector<uint8_t> tmp;
  uint8_t* host = reinterpret_cast<uint8_t*>(staging);
  if (!host) {
    tmp.assign(hi - lo, 0);
    host = tmp.data();
  } else {
    std::memset(host, 0, hi - lo);
  }
  if (n) std::memcpy(host, p->desc.data(), (size_t)n * sizeof(ImgDesc));
  std::memcpy(host + (p->off_tile_prefix - lo), p->tile_prefix.data(), (size_t)(n + 1) * 4);
  std::memcpy(host + (p->off_chunk_prefix - lo), p->chunk_prefix.data(), (size_t)(n + 1) * 4);
  std::memcpy(host + (p->off_z2_prefix - lo), p->z2_prefix.data(), (size_t)(n + 1) * 4);
  std::memcpy(host + (p->off_strip_prefix - lo), p->strip_prefix.data(), (size_t)(n + 1) * 4);
  if (p->total_wave)
    std::memcpy(host + (p->off_wave_list - lo), p->wave_list.data(), (size_t)p->total_wave * sizeof(uint2));
  if (p->total_tiles)
    std::memcpy(host + (p->off_tile_owner - lo), p->tile_owner.data(), (size_t)p->total_tiles * 4);
  if (p->total_strips)
    std::memcpy(host + (p->off_strip_owner - lo), p->strip_owner.data(), (size_t)p->total_strips * 4);
  if (cudaMemcpyAsync(base + lo, host, hi - lo, cudaMemcpyHostToDevice, st) != cudaSuccess) return RDHEI_ECUDA;
  if (!staging && cudaStreamSynchronize(st) != cudaSuccess) return RDHEI_ECUDA;   // tmp is released next
  p->ws = ws;
  Batch& B = p->batch;
  B.desc = reinterpret_cast<const ImgDesc*>(base + p->off_desc);
  B.tile_prefix = reinterpret_cast<const uint32_t*>(base + p->off_tile_prefix);
  B.chunk_prefix = reinterpret_cast<const uint32_t*>(base + p->off_chunk_prefix);
  B.z2_prefix = reinterpret_cast<const uint32_t*>(base + p->off_z2_prefix);
  B.total_z2_blocks = p->total_z2;
  B.strip_prefix = reinterpret_cast<const uint32_t*>(base + p->off_strip_prefix);
  B.tile_owner = reinterpret_cast<const uint32_t*>(base + p->off_tile_owner);
  B.strip_owner = reinterpret_cast<const uint32_t*>(base + p->off_strip_owner);
  B.total_strips = p->total_strips;
  B.n_images = n;
  B.total_tiles = p->total_tiles;
  B.total_chunks = p->total_chunks;
  B.err = reinterpret_cast<uint32_t*>(base + p->off_err);
  B.tickets = reinterpret_cast<uint32_t*>(base + p->off_tickets);
  B.hist_acc = reinterpret_cast<uint32_t*>(base + p->off_hist);
  B.chunk_status = reinterpret_cast<unsigned long long*>(base + p->off_chunk_status);
  B.tile_flags = reinterpret_cast<uint32_t*>(base + p->off_tile_flags);
  B.tile_rows = base + p->off_tile_rows;
  B.subtree = base + p->off_subtree;
  B.aux = base + p->off_aux;
  B.sigma6 = base + p->off_sigma6;
  B.tilemap = reinterpret_cast<TileMap*>(base + p->off_tilemap);
  B.lab = p->any_med ? base + p->off_lab : nullptr;
  B.wave_flags = reinterpret_cast<uint32_t*>(base + p->off_wave_flags);
  B.wave_list = reinterpret_cast<const uint2*>(base + p->off_wave_list);
  B.total_wave = p->total_wave;
  B.wave_cols = p->wave_cols;
  B.tile_cnt = reinterpret_cast<uint16_t*>(base + p->off_tile_cnt);
  B.strip_base = reinterpret_cast<uint32_t*>(base + p->off_strip_base);
  B.strip_tot = reinterpret_cast<uint32_t*>(base + p->off_strip_tot);
  B.rowcnt = base + p->off_rowcnt;
  B.part_base = reinterpret_cast<uint32_t*>(base + p->off_part_base);
  B.part_rows = TILE;
  B.count_rows = 0;
  return RDHEI_OK;
}

int rdhei_plan_upload(rdhei_plan* p, void* ws, size_t ws_bytes, void* stream) {
  return upload_impl(p, ws, ws_bytes, nullptr, 0, stream);
}

int rdhei_plan_upload_async(rdhei_plan* p, void* ws, size_t ws_bytes, void* staging, size_t staging_bytes,
                            void* stream) {
  if (!staging) return RDHEI_EINVAL;
  return upload_impl(p, ws, ws_bytes, staging, staging_bytes, stream);
}

static bool aligned4(const void* q) { return (reinterpret_cast<uintptr_t>(q) & 3) == 0; }

static int check_op(const rdhei_plan* p, int op) {
  for (const rdhei_job& j : p->jobs) {
    const bool lmr = (j.variant & 1) == RDHEI_LMR;
    switch (op) {
      case RDHEI_OP_LABEL_ENCRYPT:
        if (!j.src || !j.dst) return RDHEI_EINVAL;
        if ((j.map_bits && !aligned4(j.map_bits)) || (j.eta_bits && !aligned4(j.eta_bits))) return RDHEI_EINVAL;
        if (lmr && j.side_nbits && (!j.side_bits || !aligned4(j.side_bits))) return RDHEI_EINVAL;
        break;
      case RDHEI_OP_EMBED:
        if (!j.src || !j.dst) return RDHEI_EINVAL;
        if (j.nbits && (!j.payload || !aligned4(j.payload))) return RDHEI_EINVAL;
        if (j.nbits >= (1ull << 30)) return RDHEI_EINVAL;
        if (lmr && (!j.map_bits || !aligned4(j.map_bits))) return RDHEI_EINVAL;
        break;
      case RDHEI_OP_EXTRACT:
        if (!j.src) return RDHEI_EINVAL;
        if (j.max_bits && (!j.bits_out || !aligned4(j.bits_out))) return RDHEI_EINVAL;
        if (lmr && (!j.map_bits || !aligned4(j.map_bits))) return RDHEI_EINVAL;
        break;
      case RDHEI_OP_DECRYPT_RECOVER:
        if (!j.src || !j.dst) return RDHEI_EINVAL;
        if (lmr && (!j.map_bits || !j.eta_bits || !aligned4(j.map_bits) || !aligned4(j.eta_bits)))
          return RDHEI_EINVAL;
        break;
      case RDHEI_OP_ENCODE:
        if (!j.src || !j.dst) return RDHEI_EINVAL;
        if ((j.map_bits && !aligned4(j.map_bits)) || (j.eta_bits && !aligned4(j.eta_bits))) return RDHEI_EINVAL;
        if (lmr && j.side_nbits && (!j.side_bits || !aligned4(j.side_bits))) return RDHEI_EINVAL;
        if (lmr && !j.map_bits) return RDHEI_EINVAL;         // the hider's half reads the map back
        if (j.nbits && (!j.payload || !aligned4(j.payload))) return RDHEI_EINVAL;
        if (j.nbits >= (1ull << 30)) return RDHEI_EINVAL;
        break;
      case RDHEI_OP_DECODE:
        if (!j.src || !j.dst) return RDHEI_EINVAL;
        if (j.max_bits && (!j.bits_out || !aligned4(j.bits_out))) return RDHEI_EINVAL;
        if (lmr && (!j.map_bits || !j.eta_bits || !aligned4(j.map_bits) || !aligned4(j.eta_bits)))
          return RDHEI_EINVAL;
        break;
      case RDHEI_OP_LMR_SET_SIDE:
        if (!j.dst) return RDHEI_EINVAL;
        if (j.side_nbits && (!j.side_bits || !aligned4(j.side_bits))) return RDHEI_EINVAL;
        break;
      default:
        return RDHEI_EINVAL;
    }
  }
  return RDHEI_OK;
}

// rows of a strip per extraction CTA: the plan's setting, else whole strips unless the
// batch has fewer than four strips per SM (small batches, serving), where 16 rows
// measured fastest (one to four images of 512^2 .. 2048^2)
static int extract_rows_of(rdhei_plan* p) {
  if (p->extract_rows) return p->extract_rows;
  if (p->auto_rows) return p->auto_rows;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
      cudaSuccess || sms <= 0)
    sms = 152;
  p->auto_rows = (uint64_t)p->total_strips >= (uint64_t)sms * 4 ? TILE : 16;
  return p->auto_rows;
}

int rdhei_plan_stage_count(int op) {
  switch (op) {
    case RDHEI_OP_DECODE:
      return 5;
    case RDHEI_OP_DECRYPT_RECOVER:
      return 4;
    case RDHEI_OP_ENCODE:
    case RDHEI_OP_LABEL_ENCRYPT:
    case RDHEI_OP_EMBED:
    case RDHEI_OP_EXTRACT:
      return 3;
    case RDHEI_OP_LMR_SET_SIDE:
      return 1;
    default:
      return 0;
  }
}

const char* rdhei_stage_name(int op, int stage) {
  static const char* enc[3] = {"pass1_keystream_hist", "topmap", "enc_gather"};
  static const char* dec[4] = {"pass1_keystream_decrypt", "topmap", "dec_gather_recover", "med_wavefront"};
  static const char* fenc[3] = {"pass1_keystream_hist", "topmap_strips", "enc_gather_embed"};
  static const char* fdec[5] = {"pass1_keystream_decrypt", "topmap_strips", "extract_strips", "dec_gather_recover",
                                "med_wavefront"};
  switch (op) {
    case RDHEI_OP_ENCODE: return stage >= 0 && stage < 3 ? fenc[stage] : "";
    case RDHEI_OP_DECODE: return stage >= 0 && stage < 5 ? fdec[stage] : "";
    case RDHEI_OP_LABEL_ENCRYPT: return stage >= 0 && stage < 3 ? enc[stage] : "";
    case RDHEI_OP_DECRYPT_RECOVER: return stage >= 0 && stage < 4 ? dec[stage] : "";
    case RDHEI_OP_EMBED:
      return stage == 0 ? "z2_encrypt_count" : stage == 1 ? "embed_offsets" : stage == 2 ? "embed_scan" : "";
    case RDHEI_OP_EXTRACT:
      return stage == 0 ? "extract_count" : stage == 1 ? "extract_scan" : stage == 2 ? "z2_decrypt" : "";
    case RDHEI_OP_LMR_SET_SIDE: return stage == 0 ? "lmr_side" : "";
  }
  return "";
}

int rdhei_plan_run_stage(rdhei_plan* p, int op, int stage, void* stream) {
  if (!p || !p->ws) return RDHEI_EINVAL;
  if (stage < 0 || stage >= rdhei_plan_stage_count(op)) return RDHEI_EINVAL;
  NvtxRange range(rdhei_stage_name(op, stage));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Batch B = p->batch;
  B.part_rows = op == RDHEI_OP_DECODE ? extract_rows_of(p) : TILE;   // only the fused decode splits strips
  B.count_rows = op == RDHEI_OP_DECODE ? 1 : 0;
  if (stage == 0) {
    int rc = check_op(p, op);
    if (rc) return rc;
    uint8_t* base = reinterpret_cast<uint8_t*>(p->ws);
    if (launch_zero(base + p->off_zero, p->zero_bytes, st) != cudaSuccess) return RDHEI_ECUDA;
    if (op == RDHEI_OP_LABEL_ENCRYPT || op == RDHEI_OP_ENCODE) {
      // packed-map outputs of images whose rows do not start on a 16-bit boundary are
      // OR-ed word by word and must start from zero
      for (const rdhei_job& j : p->jobs) {
        if (j.W % 16 == 0) continue;
        const size_t bytes = (((size_t)j.H * j.W + 31) / 32) * 4;
        if (j.map_bits && cudaMemsetAsync(j.map_bits, 0, bytes, st) != cudaSuccess) return RDHEI_ECUDA;
        if ((j.variant & 1) == RDHEI_LMR && j.eta_bits && cudaMemsetAsync(j.eta_bits, 0, bytes, st) != cudaSuccess)
          return RDHEI_ECUDA;
      }
    }
  }
  switch (op) {
    case RDHEI_OP_LABEL_ENCRYPT:
      if (stage == 0) launch_pass1(B, 0, p->general, p->any_med, st);
      else if (stage == 1) launch_topmap(B, true, false, st);
      else launch_enc_pass2(B, p->any_lmr, p->any_med, (uint32_t)p->enc_split, st);
      break;
    case RDHEI_OP_EMBED:
      if (stage == 0) launch_z2_count(B, st);
      else if (stage == 1) launch_offsets(B, false, st);
      else launch_scan(B, false, st);
      break;
    case RDHEI_OP_EXTRACT:
      if (stage == 0) launch_count(B, true, st);
      else if (stage == 1) launch_scan(B, true, st);
      else launch_z2_xor(B, true, st);
      break;
    case RDHEI_OP_DECRYPT_RECOVER:
      if (stage == 0) launch_pass1(B, 1, p->general, false, st);
      else if (stage == 1) launch_topmap(B, false, false, st);
      else if (stage == 2) launch_dec_pass2(B, p->any_lmr, p->any_med, st);
      else if (p->any_med) {
        // the wavefront owns its ticket and done flags: clear them so the stage can rerun
        uint8_t* base = reinterpret_cast<uint8_t*>(p->ws);
        if (cudaMemsetAsync(base + p->off_wave_flags, 0, (size_t)p->total_wave * 4, st) != cudaSuccess ||
            cudaMemsetAsync(base + p->off_tickets + 7 * 4, 0, 4, st) != cudaSuccess)
          return RDHEI_ECUDA;
        launch_med_wave(B, st);
      }
      break;
    case RDHEI_OP_LMR_SET_SIDE:
      launch_lmr_side(B, st);
      break;
    case RDHEI_OP_ENCODE:
      if (stage == 0) launch_pass1(B, 0, p->general, p->any_med, st);
      else if (stage == 1) launch_topmap(B, true, true, st);
      else launch_enc_fused(B, p->any_lmr, p->any_med, st);
      break;
    case RDHEI_OP_DECODE:
      if (stage == 0) launch_pass1(B, 1, p->general, false, st);
      else if (stage == 1) launch_topmap(B, false, true, st);
      else if (stage == 2) launch_extract_strips(B, st);
      else if (stage == 3) launch_dec_pass2(B, p->any_lmr, p->any_med, st);
      else if (p->any_med) {
        uint8_t* base = reinterpret_cast<uint8_t*>(p->ws);
        if (cudaMemsetAsync(base + p->off_wave_flags, 0, (size_t)p->total_wave * 4, st) != cudaSuccess ||
            cudaMemsetAsync(base + p->off_tickets + 7 * 4, 0, 4, st) != cudaSuccess)
          return RDHEI_ECUDA;
        launch_med_wave(B, st);
      }
      break;
  }
  return cudaGetLastError() == cudaSuccess ? RDHEI_OK : RDHEI_ECUDA;
}

int rdhei_plan_set_wave_cols(rdhei_plan* p, int cols) {
  if (!p || p->ws || (cols != 0 && cols != 64 && cols != 128 && cols != 256)) return RDHEI_EINVAL;
  p->wave_cols = cols;
  if (layout_wave(p) != RDHEI_OK) return RDHEI_EINVAL;
  build_layout(p);
  return RDHEI_OK;
}

int rdhei_plan_set_param(rdhei_plan* p, int param, int value) {
  if (!p) return RDHEI_EINVAL;
  switch (param) {
    case RDHEI_PARAM_WAVE_COLS:
      return rdhei_plan_set_wave_cols(p, value);
    case RDHEI_PARAM_EXTRACT_ROWS:
      if (value != 0 && value != 4 && value != 8 && value != 16 && value != 32 && value != 64) return RDHEI_EINVAL;
      p->extract_rows = value;
      return RDHEI_OK;
    case RDHEI_PARAM_ENC_SPLIT:
      if (value < 0 || value > 64) return RDHEI_EINVAL;
      p->enc_split = value;
      return RDHEI_OK;
  }
  return RDHEI_EINVAL;
}

int rdhei_plan_get_param(rdhei_plan* p, int param) {
  if (!p) return -1;
  switch (param) {
    case RDHEI_PARAM_WAVE_COLS: return p->wave_cols;
    case RDHEI_PARAM_EXTRACT_ROWS: return extract_rows_of(p);
    case RDHEI_PARAM_ENC_SPLIT: return p->enc_split;
  }
  return -1;
}

int rdhei_plan_stage_active(const rdhei_plan* p, int op, int stage) {
  if (!p || stage < 0 || stage >= rdhei_plan_stage_count(op)) return 0;
  if (op == RDHEI_OP_DECRYPT_RECOVER && stage == 3) return p->any_med ? 1 : 0;
  if (op == RDHEI_OP_DECODE && stage == 4) return p->any_med ? 1 : 0;
  return 1;
}

static const char* op_range_name(int op) {
  switch (op) {
    case RDHEI_OP_LABEL_ENCRYPT: return "rdhei_label_encrypt";
    case RDHEI_OP_EMBED: return "rdhei_embed";
    case RDHEI_OP_EXTRACT: return "rdhei_extract";
    case RDHEI_OP_DECRYPT_RECOVER: return "rdhei_decrypt_recover";
    case RDHEI_OP_LMR_SET_SIDE: return "rdhei_lmr_set_side";
    case RDHEI_OP_ENCODE: return "rdhei_encode";
    case RDHEI_OP_DECODE: return "rdhei_decode";
  }
  return "rdhei_plan_run";
}

int rdhei_plan_run(rdhei_plan* p, int op, void* stream) {
  const int n = rdhei_plan_stage_count(op);
  if (n == 0) return RDHEI_EINVAL;
  NvtxRange range(op_range_name(op));
  for (int s = 0; s < n; s++) {
    int rc = rdhei_plan_run_stage(p, op, s, stream);
    if (rc) return rc;
  }
  return RDHEI_OK;
}

void rdhei_plan_destroy(rdhei_plan* p) { delete p; }

size_t rdhei_workspace_size(const rdhei_job* jobs, int n) {
  rdhei_plan* p = nullptr;
  if (rdhei_plan_create(jobs, n, &p) != RDHEI_OK) return 0;
  size_t s = p->total;
  rdhei_plan_destroy(p);
  return s;
}

static int run_once(const rdhei_job* jobs, int n, void* ws, size_t ws_bytes, void* stream, int op) {
  rdhei_plan* p = nullptr;
  int rc = rdhei_plan_create(jobs, n, &p);
  if (rc) return rc;
  rc = rdhei_plan_upload(p, ws, ws_bytes, stream);
  if (!rc) rc = rdhei_plan_run(p, op, stream);
  rdhei_plan_destroy(p);
  return rc;
}

int rdhei_label_encrypt(const rdhei_job* jobs, int n, void* ws, size_t ws_bytes, void* stream) {
  return run_once(jobs, n, ws, ws_bytes, stream, RDHEI_OP_LABEL_ENCRYPT);
}
int rdhei_embed(const rdhei_job* jobs, int n, void* ws, size_t ws_bytes, void* stream) {
  return run_once(jobs, n, ws, ws_bytes, stream, RDHEI_OP_EMBED);
}
int rdhei_extract(const rdhei_job* jobs, int n, void* ws, size_t ws_bytes, void* stream) {
  return run_once(jobs, n, ws, ws_bytes, stream, RDHEI_OP_EXTRACT);
}
int rdhei_decrypt_recover(const rdhei_job* jobs, int n, void* ws, size_t ws_bytes, void* stream) {
  return run_once(jobs, n, ws, ws_bytes, stream, RDHEI_OP_DECRYPT_RECOVER);
}
int rdhei_lmr_set_side(const rdhei_job* jobs, int n, void* ws, size_t ws_bytes, void* stream) {
  return run_once(jobs, n, ws, ws_bytes, stream, RDHEI_OP_LMR_SET_SIDE);
}
int rdhei_encode(const rdhei_job* jobs, int n, void* ws, size_t ws_bytes, void* stream) {
  return run_once(jobs, n, ws, ws_bytes, stream, RDHEI_OP_ENCODE);
}
int rdhei_decode(const rdhei_job* jobs, int n, void* ws, size_t ws_bytes, void* stream) {
  return run_once(jobs, n, ws, ws_bytes, stream, RDHEI_OP_DECODE);
}

int rdhei_workspace_status(void* ws, void* stream, int32_t* code) {
  if (!ws || !code) return RDHEI_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  uint32_t v = 0;
  if (cudaMemcpyAsync(&v, ws, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) return RDHEI_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return RDHEI_ECUDA;
  *code = (int32_t)v;
  return RDHEI_OK;
}

int rdhei_plan_copy_status(const rdhei_plan* p, int32_t* dst, void* stream) {
  if (!p || !p->ws || !dst || (reinterpret_cast<uintptr_t>(dst) & 3)) return RDHEI_EINVAL;
  const uint8_t* w = reinterpret_cast<const uint8_t*>(p->ws) + p->off_err;
  return cudaMemcpyAsync(dst, w, 4, cudaMemcpyDefault, reinterpret_cast<cudaStream_t>(stream)) == cudaSuccess
             ? RDHEI_OK : RDHEI_ECUDA;
}

size_t rdhei_job_size(void) { return sizeof(rdhei_job); }
size_t rdhei_info_size(void) { return sizeof(rdhei_info); }

const char* rdhei_version(void) { return "rdhei 0.1 sm_103a"; }

int rdhei_build_flags(void) {
#ifdef RDHEI_CHECK
  return RDHEI_BUILD_CHECKED;
#else
  return 0;
#endif
}

}  // extern "C"
