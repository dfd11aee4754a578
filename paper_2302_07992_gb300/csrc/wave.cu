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
#include "../../include/rdhei.h"
#include "common.cuh"

namespace rdhei {

constexpr int WAVE_WARPS = 4;
// spin (bounded by WAIT_LIMIT_NS from t0) until a tile's done flag is set
__device__ __forceinline__ bool wait_flag(const uint32_t* f, uint64_t t0) {
  while (ld_acquire_u32(f) == 0u) {
    if (globaltimer_ns() - t0 > WAIT_LIMIT_NS) return false;
    __nanosleep(64);
  }
  return true;
}

// labels of 64 pixels of one image row, from the tile-major de-rotated label plane
__device__ __forceinline__ uint64_t lab_row64(const Batch& B, const ImgDesc& d, int y, int x64) {
  if (x64 >= (int)d.tiles_x) return 0ull;
  const uint32_t tile = d.tile_base + (uint32_t)(y / TILE) * d.tiles_x + (uint32_t)x64;
  return *reinterpret_cast<const uint64_t*>(B.lab + (size_t)tile * AUX_BYTES + (size_t)(y % TILE) * 8);
}

template <int WCOLS>
__global__ void __launch_bounds__(32 * WAVE_WARPS) k_med_wave(Batch B) {
  constexpr int WAVE_PITCH = WCOLS + 4;
  constexpr int NLAB = WCOLS / 64;                           // 64-pixel label words per row
  __shared__ __align__(16) uint8_t tiles[WAVE_WARPS][WAVE_ROWS * WAVE_PITCH];
  __shared__ uint8_t uprow[WAVE_WARPS][WCOLS + 4];          // [0] = upper-left corner, [1 + c] = column c
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* T = tiles[warp];
  uint8_t* U = uprow[warp];
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
    uint32_t o0 = o1;                                          // my result one step earlier
    __syncwarp();

    const int y = y0 + lane;
    uint64_t lb = lab[0];
    for (int s = 0; s < cols + WAVE_ROWS - 1; s++) {
      const uint32_t bu = __shfl_up_sync(0xffffffffu, o1, 1);   // lane r-1: pixel (r-1, c)
      const uint32_t cu = __shfl_up_sync(0xffffffffu, o0, 1);   // lane r-1: pixel (r-1, c-1)
      const int c = s - lane;
      o0 = o1;
      if (lane < rows && c >= 0 && c < cols) {
        const int x = x0 + c;
        const uint32_t D = T[lane * WAVE_PITCH + c];
        const uint32_t label = (uint32_t)(lb & 1ull);
        if ((c & 63) == 63) {
          // next 64 labels: shift the words down (static register indices)
#pragma unroll
          for (int q = 0; q + 1 < NLAB; q++) lab[q] = lab[q + 1];
          lb = lab[0];
        } else {
          lb >>= 1;
        }
        uint32_t out = D;
        if (!label) {
          const uint32_t A = o1;
          const uint32_t Bv = lane > 0 ? bu : U[1 + c];
          const uint32_t C = lane > 0 ? cu : U[c];
          uint32_t pred;
          if (y == 0) pred = seven ? (A & 0xFEu) : A;            // row 0: from the left
          else if (x == 0) pred = seven ? (Bv & 0xFEu) : Bv;     // column 0: from above
          else {
            const uint32_t a = seven ? A >> 1 : A, bb = seven ? Bv >> 1 : Bv, cc = seven ? C >> 1 : C;
            const uint32_t mx = max(a, bb), mn = min(a, bb);
            const uint32_t m = cc >= mx ? mn : cc <= mn ? mx : a + bb - cc;
            pred = seven ? m << 1 : m;
          }
          out = (pred & FM) | (D & ~FM & 0xFFu);
        }
        T[lane * WAVE_PITCH + c] = (uint8_t)out;
        o1 = out;
      }
    }
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
  if (B.wave_cols == 64) launch_wave_cols<64>(B, st);
  else if (B.wave_cols == 256) launch_wave_cols<256>(B, st);
  else launch_wave_cols<128>(B, st);
}

}  // namespace rdhei
