// wave.cu -- recovery for the related-work MED variant (RDHEI_EMR_MED / RDHEI_LMR_MED):
// a label-0 pixel takes its replaced field from the median edge detector prediction of
// its RECOVERED left, upper and upper-left neighbours, so pixel (i, j) depends on every
// pixel above and to the left of it.  The recovery runs as a tiled anti-diagonal
// wavefront:
//   * tiles of 32 rows x 64, 128 or 256 columns (a plan parameter), one warp per tile,
//     lane r owns row r;
//   * inside a tile, step s recovers pixel (r, s - r) on every lane: the left value is
//     the lane's own previous result, the upper and upper-left values come from lane
//     r - 1's last two results by shuffle, so a tile takes width + 31 steps;
//   * across tiles, warps take tiles from a ticket dispenser in anti-diagonal order
//     over all images and wait (bounded) for the upper and left tiles' done flags;
//     every tile a warp waits for was handed out earlier to a running warp.
// Input: the de-rotated, decrypted image in dst (written by the gather pass) and the
// de-rotated label bits in B.lab; output: dst, recovered in place.
#include <type_traits>

#include "../../include/rdhei.h"
#include "common.cuh"

namespace rdhei {

constexpr int WAVE_WARPS = 4;
// spin (bounded by `limit` ns of %globaltimer from t0) until a tile's done flag is set
__device__ __forceinline__ bool wait_flag(const uint32_t* f, uint64_t t0, uint64_t limit = WAIT_LIMIT_NS) {
  while (ld_acquire_u32(f) == 0u) {
    if (globaltimer_ns() - t0 > limit) return false;
    __nanosleep(64);
  }
  return true;
}

// Self-test of the bounded wait: one warp waits on *flag exactly as a wavefront tile
// waits on a neighbour, then reports OK or ETIMEOUT.
__global__ void k_wait_selftest(const uint32_t* flag, uint64_t limit, int32_t* status) {
  const bool ok = wait_flag(flag, globaltimer_ns(), limit);
  if (threadIdx.x == 0) *status = ok ? 0 : ERR_TIMEOUT;
}

// labels of 64 pixels of one image row, from the tile-major de-rotated label plane
__device__ __forceinline__ uint64_t lab_row64(const Batch& B, const ImgDesc& d, int y, int x64) {
  if (x64 >= (int)d.tiles_x) return 0ull;
  const uint32_t tile = d.tile_base + (uint32_t)(y / TILE) * d.tiles_x + (uint32_t)x64;
  return *reinterpret_cast<const uint64_t*>(B.lab + (size_t)tile * AUX_BYTES + (size_t)(y % TILE) * 8);
}

template <int WCOLS>
__global__ void __launch_bounds__(32 * WAVE_WARPS) k_med_wave(Batch B) {
  // rows padded by WAVE_ROWS bytes on both sides, so that the lanes that have not
  // started or have finished read in bounds without clamping their column
  constexpr int PAD = WAVE_ROWS;
  constexpr int WAVE_PITCH = WCOLS + 2 * PAD + 4;
  constexpr int NLAB = WCOLS / 64;                           // 64-pixel label words per row
  __shared__ __align__(16) uint8_t tiles[WAVE_WARPS][WAVE_ROWS * WAVE_PITCH];
  __shared__ uint8_t uprow[WAVE_WARPS][WCOLS + 2 * PAD + 4];   // [PAD] = upper-left corner, [PAD + 1 + c] = column c
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* T = tiles[warp] + PAD;                            // T[r * WAVE_PITCH + c], c in [-PAD, WCOLS + PAD)
  uint8_t* U = uprow[warp] + PAD;
  for (;;) {
    uint32_t k = 0;
    if (lane == 0) k = atomicAdd(B.tickets + 7, 1u);
    k = __shfl_sync(0xffffffffu, k, 0);
    if (k >= B.total_wave) return;
    const uint2 e = B.wave_list[k];
    const ImgDesc& d = B.desc[e.x];
    const int ty = (int)(e.y >> 16), tx = (int)(e.y & 0xFFFFu);
    const int H = d.H, W = d.W;
    const int y0 = ty * WAVE_ROWS, x0 = tx * WCOLS;
    const int rows = min(WAVE_ROWS, H - y0), cols = min(WCOLS, W - x0);
    const rdhei_info* info = reinterpret_cast<const rdhei_info*>(d.info);
    const int b = d.b > 0 ? d.b : info->b;
    const bool lmr = d.variant == RDHEI_LMR;
    const bool seven = !lmr;
    const uint32_t FM = lmr ? (((1u << (b - 1)) - 1u) << (8 - b)) : ((0xFFu << (8 - b)) & 0xFFu);
    uint8_t* img = d.dst;

    // own tile: decrypted pixels (no other tile writes here) and my row's labels;
    // whole rows move as one 4-byte word per lane when the rows allow it
    const bool words = (W & 3) == 0 && (reinterpret_cast<uintptr_t>(img) & 3) == 0;
    if (words) {
      for (int r = 0; r < rows; r++)
        for (int c = 4 * lane; c < cols; c += 128)
          *reinterpret_cast<uint32_t*>(T + r * WAVE_PITCH + c) =
              *reinterpret_cast<const uint32_t*>(img + (size_t)(y0 + r) * W + x0 + c);
    } else {
      for (int r = 0; r < rows; r++) {
        const uint8_t* src = img + (size_t)(y0 + r) * W + x0;
        for (int c = lane; c < cols; c += 32) T[r * WAVE_PITCH + c] = src[c];
      }
    }
    uint64_t lab[NLAB];
#pragma unroll
    for (int q = 0; q < NLAB; q++) lab[q] = lane < rows ? lab_row64(B, d, y0 + lane, x0 / 64 + q) : 0ull;

    // wait for the upper and left tiles (their own dependencies are then done too)
    if (lane == 0) {
      const uint64_t t0 = globaltimer_ns();
      bool ok = true;
      if (ty > 0) ok = wait_flag(B.wave_flags + d.wave_base + (uint32_t)(ty - 1) * d.wave_tx + tx, t0) && ok;
      if (tx > 0) ok = wait_flag(B.wave_flags + d.wave_base + (uint32_t)ty * d.wave_tx + tx - 1, t0) && ok;
      if (!ok) set_error(B.err, ERR_TIMEOUT);         // outputs invalid; carry on so no wait chains up
    }
    __syncwarp();

    // borders from the recovered neighbours: the row above (with its left corner) and
    // the column to the left; L2 loads, written by other warps
    if (ty > 0) {
      const uint8_t* ur = img + (size_t)(y0 - 1) * W + x0;
      for (int c = lane; c < cols; c += 32) U[1 + c] = __ldcg(ur + c);
      if (lane == 0) U[0] = tx > 0 ? __ldcg(ur - 1) : (uint8_t)0;
    }
    uint32_t o1 = 0;                                           // my last result (left of the next pixel)
    if (tx > 0 && lane < rows) o1 = __ldcg(img + (size_t)(y0 + lane) * W + x0 - 1);
    uint32_t cprev = __shfl_up_sync(0xffffffffu, o1, 1);       // upper-left of my first pixel
    __syncwarp();

    // one pixel per lane and step, branch-free: the only dependency between steps is
    // the shuffle of lane r - 1's last result (the upper value; the upper-left one is
    // the upper value of the step before).  EMR predicts on the top seven bits: the
    // median of the values with the LSB cleared is twice the median of the seven-bit
    // values.  Tiles on the image's top row or left column also apply the border rules.
    const int y = y0 + lane;
    const uint32_t keep = seven ? 0xFEu : 0xFFu;
    const uint32_t FMc = ~FM & 0xFFu;
    uint64_t lb = lab[0];
    auto run = [&](auto border) {
      for (int s = 0; s < cols + WAVE_ROWS - 1; s++) {
        const uint32_t bu = __shfl_up_sync(0xffffffffu, o1, 1);   // lane r-1: pixel (r-1, c)
        const int c = s - lane;                                    // in [-31, cols + 30]: padded
        const uint32_t D = T[lane * WAVE_PITCH + c];
        const uint32_t Bv = lane > 0 ? bu : (uint32_t)U[1 + c];
        const uint32_t Cv = lane > 0 ? cprev : (uint32_t)U[c];
        cprev = bu;
        const uint32_t a = o1 & keep, bb = Bv & keep, cv = Cv & keep;
        const uint32_t mn = min(a, bb), mx = max(a, bb);
        uint32_t pred = mn + mx - min(max(cv, mn), mx);          // MED = min + max - clamp(C)
        if (decltype(border)::value) {
          pred = (x0 + c == 0) ? (Bv & keep) : pred;             // column 0: from above
          pred = (y == 0) ? (o1 & keep) : pred;                   // row 0: from the left
        }
        const uint32_t out = (lb & 1ull) ? D : ((pred & FM) | (D & FMc));
        if (lane < rows && c >= 0 && c < cols) {
          T[lane * WAVE_PITCH + c] = (uint8_t)out;
          o1 = out;
          if ((c & 63) == 63) {
            // next 64 labels: shift the words down (static register indices)
#pragma unroll
            for (int q = 0; q + 1 < NLAB; q++) lab[q] = lab[q + 1];
            lb = lab[0];
          } else {
            lb >>= 1;
          }
        }
      }
    };
    if (ty == 0 || tx == 0) run(std::true_type{});
    else run(std::false_type{});
    __syncwarp();
    if (words) {
      for (int r = 0; r < rows; r++)
        for (int c = 4 * lane; c < cols; c += 128)
          *reinterpret_cast<uint32_t*>(img + (size_t)(y0 + r) * W + x0 + c) =
              *reinterpret_cast<const uint32_t*>(T + r * WAVE_PITCH + c);
    } else {
      for (int r = 0; r < rows; r++) {
        uint8_t* dst = img + (size_t)(y0 + r) * W + x0;
        for (int c = lane; c < cols; c += 32) dst[c] = T[r * WAVE_PITCH + c];
      }
    }
    __syncwarp();
    if (lane == 0) {
      __threadfence();
      st_release_u32(B.wave_flags + d.wave_base + (uint32_t)ty * d.wave_tx + tx, 1u);
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------------
// Row-band pipeline (wave_cols = 0).  One CTA per image at a time (ticket dispenser
// over the MED images), BAND_WARPS warps; warp w recovers the 32-row bands w,
// w + BAND_WARPS, ...  Lane r owns row r of its band and step s recovers column s - r,
// so a band is one continuous wavefront of W + 31 steps.  A band only needs the last
// row of the band above, so it runs a few dozen steps behind it instead of a whole
// tile behind: the image's critical path is about W + 48 * bands steps.
//   * Inside a round the edge row goes from warp w to warp w + 1 through a shared ring
//     of RING bytes, with monotonic produced / consumed counters checked every
//     BAND_G steps (the producer may run at most RING columns ahead).
//   * The first band of the next round reads the previous round's last band from the
//     image itself, published per stored 64-column chunk (no back-pressure, so the
//     wait graph has no cycle).
//   * Pixels, labels (and, for the first band of a round, the row above) are staged in
//     shared memory by 64-column chunks, double-buffered; a chunk is written back and
//     its buffer refilled once every lane has passed it.
// Every wait is bounded by WAIT_LIMIT_NS, after which the error word is set and the
// warp carries on (outputs invalid, no hang).
// ---------------------------------------------------------------------------------
constexpr int BAND_WARPS = 16;
constexpr int BAND_CH = 64;            // staged columns per chunk
constexpr int BAND_G = 16;             // steps between counter checks
constexpr int RING = 256;              // edge-row ring per channel (power of two)
constexpr int BAND_PITCH = BAND_CH + 4;   // staged row pitch: the diagonal of a step hits 32 banks

struct BandSmem {
  uint8_t px[BAND_WARPS][2][WAVE_ROWS][BAND_PITCH];   // staged pixels, recovered in place
  uint64_t lab[BAND_WARPS][2][WAVE_ROWS];             // label words of the staged chunks
  uint8_t up[BAND_WARPS][2][BAND_CH + 4];             // [0] = column 64k - 1, [1 + j] = column 64k + j
  uint8_t ring[BAND_WARPS][RING];                     // edge row of warp w's band, for warp w + 1
  volatile uint32_t produced[BAND_WARPS], consumed[BAND_WARPS];
  volatile uint32_t wrap_stored;                      // columns of the round's last band in the image
  uint32_t img;
};

__device__ __forceinline__ bool band_wait_ge(volatile uint32_t* v, uint32_t target, uint32_t* err) {
  if (*v >= target) return true;
  const uint64_t t0 = globaltimer_ns();
  while (*v < target) {
    if (globaltimer_ns() - t0 > WAIT_LIMIT_NS) { set_error(err, ERR_TIMEOUT); return false; }
    __nanosleep(32);
  }
  return true;
}

__global__ void __launch_bounds__(32 * BAND_WARPS, 2) k_med_band(Batch B) {
  extern __shared__ __align__(16) uint8_t band_smem[];
  BandSmem& S = *reinterpret_cast<BandSmem*>(band_smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      S.img = atomicAdd(B.tickets + 7, 1u);
      S.wrap_stored = 0;
    }
    if (threadIdx.x < BAND_WARPS) { S.produced[threadIdx.x] = 0; S.consumed[threadIdx.x] = 0; }
    __syncthreads();
    if (S.img >= B.total_wave) return;
    const ImgDesc& d = B.desc[B.wave_list[S.img].x];
    const int H = d.H, W = d.W;
    const rdhei_info* info = reinterpret_cast<const rdhei_info*>(d.info);
    const int b = d.b > 0 ? d.b : info->b;
    const bool lmr = d.variant == RDHEI_LMR;
    const uint32_t FM = lmr ? (((1u << (b - 1)) - 1u) << (8 - b)) : ((0xFFu << (8 - b)) & 0xFFu);
    uint8_t* img = d.dst;
    const int nb = (H + WAVE_ROWS - 1) / WAVE_ROWS;
    const int nch = (W + BAND_CH - 1) / BAND_CH;
    const bool words = (W & 3) == 0 && (reinterpret_cast<uintptr_t>(img) & 3) == 0;

    for (int band = warp; band < nb; band += BAND_WARPS) {
      const int y0 = band * WAVE_ROWS, rows = min(WAVE_ROWS, H - y0);
      const uint32_t k = (uint32_t)(band / BAND_WARPS);             // round
      const uint32_t seq0 = k * (uint32_t)W;                        // channel sequence base
      const bool wrap_in = band > 0 && warp == 0;                   // upper band: previous round
      const bool ring_in = band > 0 && warp > 0;
      const bool ring_out = band + 1 < nb && warp + 1 < BAND_WARPS;
      const bool wrap_out = band + 1 < nb && warp + 1 == BAND_WARPS;

      // stage chunk q into buffer q & 1: pixels, label words and (first band of a
      // round) the row above, once the previous round's last band has stored it
      auto stage = [&](int q) {
        const int c0 = q * BAND_CH, cols = min(BAND_CH, W - c0), bi = q & 1;
        if (wrap_in) {
          band_wait_ge(&S.wrap_stored, (k - 1) * (uint32_t)W + (uint32_t)(c0 + cols), B.err);
          __threadfence_block();
          const uint8_t* ur = img + (size_t)(y0 - 1) * W;
          for (int j = lane; j < cols; j += 32) S.up[warp][bi][1 + j] = __ldcg(ur + c0 + j);
          if (lane == 0) S.up[warp][bi][0] = c0 > 0 ? __ldcg(ur + c0 - 1) : (uint8_t)0;
        }
        if (words) {
          for (int i = lane; i < rows * (BAND_CH / 4); i += 32) {
            const int r = i / (BAND_CH / 4), c = 4 * (i % (BAND_CH / 4));
            if (c < cols)
              *reinterpret_cast<uint32_t*>(&S.px[warp][bi][r][c]) =
                  *reinterpret_cast<const uint32_t*>(img + (size_t)(y0 + r) * W + c0 + c);
          }
        } else {
          for (int i = lane; i < rows * BAND_CH; i += 32) {
            const int r = i / BAND_CH, c = i % BAND_CH;
            if (c < cols) S.px[warp][bi][r][c] = img[(size_t)(y0 + r) * W + c0 + c];
          }
        }
        if (lane < rows) S.lab[warp][bi][lane] = lab_row64(B, d, y0 + lane, q);
      };
      // write chunk q back to the image
      auto store = [&](int q) {
        const int c0 = q * BAND_CH, cols = min(BAND_CH, W - c0), bi = q & 1;
        if (words) {
          for (int i = lane; i < rows * (BAND_CH / 4); i += 32) {
            const int r = i / (BAND_CH / 4), c = 4 * (i % (BAND_CH / 4));
            if (c < cols)
              *reinterpret_cast<uint32_t*>(img + (size_t)(y0 + r) * W + c0 + c) =
                  *reinterpret_cast<const uint32_t*>(&S.px[warp][bi][r][c]);
          }
        } else {
          for (int i = lane; i < rows * BAND_CH; i += 32) {
            const int r = i / BAND_CH, c = i % BAND_CH;
            if (c < cols) img[(size_t)(y0 + r) * W + c0 + c] = S.px[warp][bi][r][c];
          }
        }
      };
      stage(0);
      if (nch > 1) stage(1);
      __syncwarp();

      const int y = y0 + lane;
      const int T = W + WAVE_ROWS - 1;
      uint32_t o1 = 0, o0 = 0;                  // my last two results
      uint64_t lb = 0;
      int next_store = 0;
      for (int s0 = 0; s0 < T; s0 += BAND_G) {
        // the band above must have produced the columns lane 0 reads in this block; the
        // band below must have consumed the ring slots lane 31 overwrites
        if (ring_in) band_wait_ge(&S.produced[warp - 1], seq0 + (uint32_t)min(s0 + BAND_G, W), B.err);
        if (ring_out) {
          // slot (seq0 + c) & (RING - 1) last held column seq0 + c - RING of this channel,
          // possibly of the previous round's band
          const int last = min(s0 - (WAVE_ROWS - 1) + BAND_G, W);
          const int64_t need = (int64_t)seq0 + last - RING;
          if (last > 0 && need > 0) band_wait_ge(&S.consumed[warp], (uint32_t)need, B.err);
        }
        __syncwarp();
        __threadfence_block();
#pragma unroll 4
        for (int j = 0; j < BAND_G; j++) {
          const int s = s0 + j;
          const uint32_t bu = __shfl_up_sync(0xffffffffu, o1, 1);   // lane r-1: pixel (r-1, c)
          const uint32_t cu = __shfl_up_sync(0xffffffffu, o0, 1);   // lane r-1: pixel (r-1, c-1)
          const int c = s - lane;
          o0 = o1;
          if (lane < rows && c >= 0 && c < W) {
            const int bi = (c >> 6) & 1, cc = c & (BAND_CH - 1);
            if (cc == 0) lb = S.lab[warp][bi][lane];
            const uint32_t D = S.px[warp][bi][lane][cc];
            uint32_t out = D;
            if (!(lb & 1ull)) {
              const uint32_t A = o1;
              uint32_t Bv, C;
              if (lane > 0) { Bv = bu; C = cu; }
              else if (ring_in) {
                Bv = S.ring[warp - 1][(seq0 + (uint32_t)c) & (RING - 1)];
                C = S.ring[warp - 1][(seq0 + (uint32_t)c - 1u) & (RING - 1)];
              } else if (wrap_in) {
                Bv = S.up[warp][bi][1 + cc];
                C = S.up[warp][bi][cc];
              } else { Bv = 0; C = 0; }
              uint32_t pred;
              if (y == 0) pred = lmr ? A : (A & 0xFEu);                 // row 0: from the left
              else if (c == 0) pred = lmr ? Bv : (Bv & 0xFEu);          // column 0: from above
              else {
                const uint32_t a = lmr ? A : A >> 1, bb = lmr ? Bv : Bv >> 1, cc2 = lmr ? C : C >> 1;
                const uint32_t mx = max(a, bb), mn = min(a, bb);
                const uint32_t m = cc2 >= mx ? mn : cc2 <= mn ? mx : a + bb - cc2;
                pred = lmr ? m : m << 1;
              }
              out = (pred & FM) | (D & ~FM & 0xFFu);
            }
            lb >>= 1;
            S.px[warp][bi][lane][cc] = (uint8_t)out;
            if (ring_out && lane == WAVE_ROWS - 1) S.ring[warp][(seq0 + (uint32_t)c) & (RING - 1)] = (uint8_t)out;
            o1 = out;
          }
        }
        __syncwarp();
        __threadfence_block();
        const int s_end = min(s0 + BAND_G, T);
        if (lane == 0) {
          if (ring_out) S.produced[warp] = seq0 + (uint32_t)max(0, min(s_end - (WAVE_ROWS - 1), W));
          if (ring_in) S.consumed[warp - 1] = seq0 + (uint32_t)min(s_end, W);
        }
        // chunks every lane has passed: write back, refill the buffer with chunk + 2
        const int cdone = min(s_end - rows, W - 1);   // last column finished by every row
        while (next_store < nch && min((next_store + 1) * BAND_CH, W) - 1 <= cdone) {
          store(next_store);
          __syncwarp();
          if (wrap_out) {
            __threadfence_block();
            if (lane == 0) S.wrap_stored = seq0 + (uint32_t)min((next_store + 1) * BAND_CH, W);
          }
          if (next_store + 2 < nch) stage(next_store + 2);
          __syncwarp();
          next_store++;
        }
      }
      if (lane == 0) {
        if (ring_out) S.produced[warp] = seq0 + (uint32_t)W;
        if (ring_in) S.consumed[warp - 1] = seq0 + (uint32_t)W;
      }
    }
    __threadfence();                             // the image's pixels are out before the next image
  }
}

template <int WCOLS>
static void launch_wave_cols(const Batch& B, cudaStream_t st) {
  int dev = 0, sms = 1, occ = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_med_wave<WCOLS>, 32 * WAVE_WARPS, 0);
  uint32_t grid = (uint32_t)(sms * (occ > 0 ? occ : 1));
  const uint32_t need = (B.total_wave + WAVE_WARPS - 1) / WAVE_WARPS;     // one tile per warp at least
  if (grid > need) grid = need;
  k_med_wave<WCOLS><<<grid, 32 * WAVE_WARPS, 0, st>>>(B);
}

void launch_med_wave(const Batch& B, cudaStream_t st) {
  if (B.total_wave == 0) return;
  if (B.wave_cols == 0) {
    const int smem = (int)sizeof(BandSmem);
    cudaFuncSetAttribute(k_med_band, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int dev = 0, sms = 1, occ = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_med_band, 32 * BAND_WARPS, smem);
    uint32_t grid = (uint32_t)(sms * (occ > 0 ? occ : 1));
    if (grid > B.total_wave) grid = B.total_wave;
    k_med_band<<<grid, 32 * BAND_WARPS, smem, st>>>(B);
    return;
  }
  if (B.wave_cols == 64) launch_wave_cols<64>(B, st);
  else if (B.wave_cols == 256) launch_wave_cols<256>(B, st);
  else launch_wave_cols<128>(B, st);
}

}  // namespace rdhei

extern "C" int rdhei_wait_selftest(const uint32_t* flag, uint64_t limit_ns, int32_t* status, void* stream) {
  if (!flag || !status || (reinterpret_cast<uintptr_t>(flag) & 3) || (reinterpret_cast<uintptr_t>(status) & 3))
    return RDHEI_EINVAL;
  if (limit_ns > rdhei::WAIT_LIMIT_NS) limit_ns = rdhei::WAIT_LIMIT_NS;
  rdhei::k_wait_selftest<<<1, 32, 0, reinterpret_cast<cudaStream_t>(stream)>>>(flag, limit_ns, status);
  return cudaGetLastError() == cudaSuccess ? RDHEI_OK : RDHEI_ECUDA;
}
