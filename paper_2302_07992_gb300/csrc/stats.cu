// stats.cu -- security and quality statistics for batches of images: Shannon entropy
// and the chi-square statistic of an image's grey-level histogram, NPCR, UACI and PSNR
// between two images (Sec. IV-C, Tab. analysis), and SSIM (Wang et al. 2004), which
// the paper reports for reconstructed images (Sec. IV).
//
// k_stats: one pass over the pixels.  Each CTA takes 8192 pixels of one image, builds
// per-warp shared histograms and the pair sums (pixels that differ, sum |a - b|,
// sum (a - b)^2) and adds them into the image's accumulators; the last CTA of an
// image turns the accumulators into the fp64 metrics.
//
// k_ssim: an 11 x 11 separable Gaussian stencil.  A CTA owns 64 x 32 window positions;
// it stages the (64 + 10) x (32 + 10) input pixels of both images in shared memory,
// runs the horizontal 11-tap pass over all 42 rows into four shared planes (mu_a, mu_b,
// E[a^2 + b^2], E[ab], pixels centred at 128), then the vertical pass with eight
// outputs per thread, combines the local moments into the SSIM of each window and
// adds the window sum into the image's fp64 accumulator.  The last CTA of an image
// writes the mean.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/rdhei.h"
#include "common.cuh"

namespace rdhei {

constexpr int ST_THREADS = 256;
constexpr int ST_PX = 8192;              // pixels per k_stats CTA
// per-image accumulator words: hist[256], n_diff, stats_done, sum_abs (u64), sum_sq (u64),
// ssim_done, pad, ssim_sum (f64), pad to 272 words (8-byte aligned per image)
constexpr int ST_ACC_WORDS = 272;
constexpr int ACC_NDIFF = 256, ACC_DONE = 257, ACC_ABS = 258, ACC_SQ = 260, ACC_SSIM_DONE = 262, ACC_SSIM = 264;

constexpr int SS_K = 11;                 // window side
constexpr int SS_TX = 64, SS_TY = 32;    // window positions per CTA
constexpr int SS_INY = SS_TY + SS_K - 1;   // 42 input rows (of SS_TX + 10 = 74 columns)
constexpr int SS_PITCH = 80;             // bytes per staged input row (16-byte multiple, >= 74)
constexpr int SS_SEG = 8;                // horizontal outputs per item, vertical outputs per thread
constexpr int SS_HITEMS = SS_INY * (SS_TX / SS_SEG);   // 336 horizontal items
constexpr int SS_SMEM = 4 * SS_INY * SS_PITCH + 4 * SS_INY * SS_TX * 4;   // 56448 bytes: two input buffers

struct StatsDesc {
  const uint8_t* a;
  const uint8_t* b;
  rdhei_stats* out;
  uint64_t npx;
  int32_t H, W;
  uint32_t chunk_base, nchunks;
  uint32_t ss_base, ss_tiles_x, ss_ntiles, want_ssim;
};

struct StatsBatch {
  const StatsDesc* desc;
  const uint32_t* chunk_prefix;        // n + 1 entries
  const uint32_t* ss_prefix;           // n + 1 entries
  int n;
  uint32_t total_chunks, total_ss_tiles;
  uint32_t* acc;                       // n * ST_ACC_WORDS, zeroed per call
  float g[SS_K];                       // normalised 1-D Gaussian, sigma 1.5
};

__device__ __forceinline__ float centred(uint32_t word, int k) {
  // byte k of word as a float minus 128: 2^23 + byte assembled by one byte permute
  const uint32_t sel = (uint32_t)k | 0x7540u;
  return __int_as_float((int)__byte_perm(word, 0x4B000000u, sel)) - 8388736.0f;
}

// ---------------------------------------------------------------- k_stats --
// Persistent: CTA c owns the contiguous chunk range [c * per, (c + 1) * per), so most
// of its chunks belong to one image.  Counts stay in shared memory across the chunks
// of an image and go to the image's global accumulators once per image run; the CTA
// whose run completes the image's chunk count writes the metrics.
struct StatsSmem {
  uint32_t h[ST_THREADS / 32][256];
  double red_h[ST_THREADS / 32], red_c[ST_THREADS / 32];
  unsigned long long abs_sum, sq_sum;
  uint32_t ndiff, last;
};

__device__ void stats_flush(const StatsBatch& B, int img, uint32_t run, StatsSmem& S) {
  const int t = threadIdx.x;
  const StatsDesc& d = B.desc[img];
  uint32_t* acc = B.acc + (size_t)img * ST_ACC_WORDS;
  __syncthreads();
  for (int v = t; v < 256; v += ST_THREADS) {
    uint32_t c = 0;
#pragma unroll
    for (int w = 0; w < ST_THREADS / 32; w++) { c += S.h[w][v]; S.h[w][v] = 0; }
    if (c) atomicAdd(acc + v, c);
  }
  __syncthreads();
  if (t == 0) {
    atomicAdd(acc + ACC_NDIFF, S.ndiff);
    atomicAdd(reinterpret_cast<unsigned long long*>(acc + ACC_ABS), S.abs_sum);
    atomicAdd(reinterpret_cast<unsigned long long*>(acc + ACC_SQ), S.sq_sum);
    S.ndiff = 0; S.abs_sum = 0; S.sq_sum = 0;
    __threadfence();
    S.last = atomicAdd(acc + ACC_DONE, run) + run == d.nchunks;
  }
  __syncthreads();
  if (!S.last) return;
  __threadfence();
  // one bin per thread: the fp64 logarithms run on all warps, then a block sum
  rdhei_stats* out = d.out;
  const double N = (double)d.npx;
  double th = 0.0, tc = 0.0;
  for (int v = t; v < 256; v += ST_THREADS) {
    const uint32_t c = __ldcg(acc + v);
    out->hist[v] = c;
    const double P = (double)c / N;
    if (c) th -= P * log2(P);
    tc += (P - 1.0 / 256.0) * (P - 1.0 / 256.0);
  }
  for (int off = 16; off; off >>= 1) {
    th += __shfl_xor_sync(0xffffffffu, th, off);
    tc += __shfl_xor_sync(0xffffffffu, tc, off);
  }
  if ((t & 31) == 0) { S.red_h[t >> 5] = th; S.red_c[t >> 5] = tc; }
  __syncthreads();
  if (t == 0) {
    double H = 0.0, chi = 0.0;
    for (int w = 0; w < ST_THREADS / 32; w++) { H += S.red_h[w]; chi += S.red_c[w]; }
    const uint64_t nd = __ldcg(acc + ACC_NDIFF);
    const uint64_t sa = __ldcg(reinterpret_cast<const unsigned long long*>(acc + ACC_ABS));
    const uint64_t sq = __ldcg(reinterpret_cast<const unsigned long long*>(acc + ACC_SQ));
    out->n_diff = nd;
    out->sum_abs = sa;
    out->sum_sq = sq;
    out->entropy = H;
    out->chi2 = 256.0 * N * chi;
    if (d.b) {
      out->npcr = 100.0 * (double)nd / N;
      out->uaci = 100.0 * (double)sa / (255.0 * N);
      out->psnr = sq ? 10.0 * log10(255.0 * 255.0 * N / (double)sq) : (double)INFINITY;
    } else {
      out->npcr = out->uaci = out->psnr = (double)NAN;
    }
    if (!d.want_ssim) out->ssim = (double)NAN;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(ST_THREADS) k_stats(StatsBatch B) {
  __shared__ StatsSmem S;
  const int t = threadIdx.x, warp = t >> 5;
  for (int i = t; i < (ST_THREADS / 32) * 256; i += ST_THREADS) (&S.h[0][0])[i] = 0u;
  if (t == 0) { S.abs_sum = 0; S.sq_sum = 0; S.ndiff = 0; }
  const uint32_t per = (B.total_chunks + gridDim.x - 1) / gridDim.x;
  const uint32_t g0 = blockIdx.x * per, g1 = umin64((uint64_t)g0 + per, B.total_chunks);
  if (g0 >= g1) return;
  int img = owner_of(B.chunk_prefix, B.n, g0);
  uint32_t run = 0;
  __syncthreads();
  for (uint32_t g = g0; g < g1; g++) {
    while (g >= __ldg(B.chunk_prefix + img + 1)) {   // next image (empty images have no chunks)
      if (run) stats_flush(B, img, run, S);
      run = 0;
      img++;
    }
    const StatsDesc& d = B.desc[img];
    const uint64_t p0 = (uint64_t)(g - d.chunk_base) * ST_PX + 32ull * t;
    const int valid = p0 < d.npx ? (int)umin64(32, d.npx - p0) : 0;
    uint32_t ndiff = 0, sabs = 0, ssq = 0;
    if (valid > 0) {
      uint32_t wa[8], wb[8];
      const uint8_t* pa = d.a + p0;
      const uint8_t* pb = d.b ? d.b + p0 : nullptr;
      const bool vec = valid == 32 && ((reinterpret_cast<uintptr_t>(pa) & 15) == 0) &&
                       (!pb || ((reinterpret_cast<uintptr_t>(pb) & 15) == 0));
#pragma unroll
      for (int i = 0; i < 8; i++) { wa[i] = 0; wb[i] = 0; }
      if (vec) {
        const uint4 a0 = __ldcs(reinterpret_cast<const uint4*>(pa)), a1 = __ldcs(reinterpret_cast<const uint4*>(pa) + 1);
        wa[0] = a0.x; wa[1] = a0.y; wa[2] = a0.z; wa[3] = a0.w; wa[4] = a1.x; wa[5] = a1.y; wa[6] = a1.z; wa[7] = a1.w;
        if (pb) {
          const uint4 b0 = __ldcs(reinterpret_cast<const uint4*>(pb)), b1 = __ldcs(reinterpret_cast<const uint4*>(pb) + 1);
          wb[0] = b0.x; wb[1] = b0.y; wb[2] = b0.z; wb[3] = b0.w; wb[4] = b1.x; wb[5] = b1.y; wb[6] = b1.z; wb[7] = b1.w;
        }
      } else {
#pragma unroll
        for (int k = 0; k < 32; k++) {
          if (k < valid) {
            wa[k >> 2] |= (uint32_t)pa[k] << (8 * (k & 3));
            if (pb) wb[k >> 2] |= (uint32_t)pb[k] << (8 * (k & 3));
          }
        }
      }
#pragma unroll
      for (int k = 0; k < 32; k++)
        if (k < valid) atomicAdd(&S.h[warp][(wa[k >> 2] >> (8 * (k & 3))) & 0xFFu], 1u);
      if (pb) {
        // four pixels at a time; bytes past `valid` are zero in both words
#pragma unroll
        for (int w = 0; w < 8; w++) {
          const uint32_t dd = __vabsdiffu4(wa[w], wb[w]);
          sabs = __dp4a(dd, 0x01010101u, sabs);
          ssq = __dp4a(dd, dd, ssq);
          ndiff += __popc((((dd & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | dd) & 0x80808080u);
        }
      }
    }
    // warp sums fit 32 bits: at most 32 lanes x 32 pixels x 255^2
    if (d.b) {
      ndiff = __reduce_add_sync(0xffffffffu, ndiff);
      sabs = __reduce_add_sync(0xffffffffu, sabs);
      ssq = __reduce_add_sync(0xffffffffu, ssq);
      if ((t & 31) == 0) {
        atomicAdd(&S.ndiff, ndiff);
        atomicAdd(&S.abs_sum, (unsigned long long)sabs);
        atomicAdd(&S.sq_sum, (unsigned long long)ssq);
      }
    }
    run++;
  }
  stats_flush(B, img, run, S);
}

// ----------------------------------------------------------------- k_ssim --
// Position of 16-byte chunk q (two float2 columns) of a 64-column float2 row: the four
// chunks of a horizontal item are rotated by (item segment / 2), so that the 8 items of
// a row store their chunks to 8 different bank groups; readers of one column pair
// undo the same rotation.
__device__ __forceinline__ int swz_chunk(int q) { return (q & ~3) | (((q & 3) + (q >> 3)) & 3); }

// two independent IEEE fp32 fused multiply-adds (round to nearest) in one instruction
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  unsigned long long pa, pb, pc, r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(pa) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(pb) : "f"(b.x), "f"(b.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(pc) : "f"(c.x), "f"(c.y));
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(pa), "l"(pb), "l"(pc));
  float2 o;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(o.x), "=f"(o.y) : "l"(r));
  return o;
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src, int bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(bytes) : "memory");
}
// (cp_async_commit / cp_async_wait_all: common.cuh)

// Stage the (SS_TY + 10) x SS_PITCH input rectangle of both images for one tile.
// 16-byte or 4-byte asynchronous copies when the rows allow it (zero-filled outside
// the image), plain byte loads otherwise.  Zeros outside the image feed only window
// positions that are masked out.
__device__ __forceinline__ void ssim_stage(const StatsDesc& d, int x0, int y0, uint8_t* ta, uint8_t* tb) {
  const int t = threadIdx.x, H = d.H, W = d.W;
  const uintptr_t align = reinterpret_cast<uintptr_t>(d.a) | reinterpret_cast<uintptr_t>(d.b);
  if ((W & 15) == 0 && (align & 15) == 0) {
    constexpr int CPR = SS_PITCH / 16;                       // 5 chunks per staged row
    for (int i = t; i < 2 * SS_INY * CPR; i += ST_THREADS) {
      const int img = i >= SS_INY * CPR, j = i - img * SS_INY * CPR;
      const int r = j / CPR, c = (j - r * CPR) * 16;
      const int y = y0 + r, x = x0 + c;
      const bool in = y < H && x < W;
      const uint8_t* base = img ? d.b : d.a;
      cp_async16((img ? tb : ta) + r * SS_PITCH + c, in ? base + (size_t)y * W + x : base, in ? 16 : 0);
    }
  } else if ((W & 3) == 0 && (align & 3) == 0) {
    constexpr int WPR = SS_PITCH / 4;
    for (int i = t; i < 2 * SS_INY * WPR; i += ST_THREADS) {
      const int img = i >= SS_INY * WPR, j = i - img * SS_INY * WPR;
      const int r = j / WPR, c = (j - r * WPR) * 4;
      const int y = y0 + r, x = x0 + c;
      const bool in = y < H && x < W;
      const uint8_t* base = img ? d.b : d.a;
      cp_async4((img ? tb : ta) + r * SS_PITCH + c, in ? base + (size_t)y * W + x : base, in ? 4 : 0);
    }
  } else {
    for (int i = t; i < SS_INY * SS_PITCH; i += ST_THREADS) {
      const int r = i / SS_PITCH, c = i - r * SS_PITCH;
      const int y = y0 + r, x = x0 + c;
      uint8_t va = 0, vb = 0;
      if (y < H && x < W) {
        const size_t o = (size_t)y * W + x;
        va = __ldg(d.a + o);
        vb = __ldg(d.b + o);
      }
      ta[r * SS_PITCH + c] = va;
      tb[r * SS_PITCH + c] = vb;
    }
  }
}

// Adds a run of `run` tiles of image img (window sum in s_sum) to the image's
// accumulators; the CTA that completes the image's tile count writes the mean.
// Called by all threads after a barrier that follows the run's last s_sum update.
__device__ void ssim_flush(const StatsBatch& B, int img, uint32_t run, double& s_sum) {
  if (threadIdx.x == 0) {
    const StatsDesc& d = B.desc[img];
    uint32_t* acc = B.acc + (size_t)img * ST_ACC_WORDS;
    atomicAdd(reinterpret_cast<double*>(acc + ACC_SSIM), s_sum);
    s_sum = 0.0;
    __threadfence();
    if (atomicAdd(acc + ACC_SSIM_DONE, run) + run == d.ss_ntiles) {
      __threadfence();
      const double sum = __ldcg(reinterpret_cast<const double*>(acc + ACC_SSIM));
      d.out->ssim = sum / ((double)(d.H - SS_K + 1) * (double)(d.W - SS_K + 1));
    }
  }
}

// Persistent over a contiguous range of tiles; the next tile's pixels are copied into
// the second input buffer while the current tile is computed.
__global__ void __launch_bounds__(ST_THREADS, 3) k_ssim(StatsBatch B) {
  extern __shared__ __align__(16) uint8_t smem[];
  constexpr int IN_BYTES = 2 * SS_INY * SS_PITCH;           // a and b rectangles
  uint8_t* tin0 = smem;
  uint8_t* tin1 = smem + IN_BYTES;
  // horizontal results, two float2 planes: (mu_a, mu_b) and (E[a^2 + b^2], E[ab])
  float2* h_ab = reinterpret_cast<float2*>(smem + 2 * IN_BYTES);   // [SS_INY][SS_TX]
  float2* h_q = h_ab + SS_INY * SS_TX;
  __shared__ double s_sum;
  const int t = threadIdx.x;
  const uint32_t G = B.total_ss_tiles;
  // CTA c owns the contiguous tiles [c * per, (c + 1) * per): the image changes rarely
  const uint32_t per = (G + gridDim.x - 1) / gridDim.x;
  const uint32_t gbeg = blockIdx.x * per, gend = umin64((uint64_t)gbeg + per, G);
  if (gbeg >= gend) return;
  if (t == 0) s_sum = 0.0;
  float2 g2[SS_K];
#pragma unroll
  for (int k = 0; k < SS_K; k++) g2[k] = make_float2(B.g[k], B.g[k]);
  const float2 off2 = make_float2(-8388736.0f, -8388736.0f);
  int img = owner_of(B.ss_prefix, B.n, gbeg);
  uint32_t img_end = __ldg(B.ss_prefix + img + 1);
  {
    const StatsDesc& d = B.desc[img];
    const uint32_t tile = gbeg - d.ss_base;
    ssim_stage(d, (int)(tile % d.ss_tiles_x) * SS_TX, (int)(tile / d.ss_tiles_x) * SS_TY, tin0, tin0 + SS_INY * SS_PITCH);
    cp_async_commit();
  }
  int cur = 0;
  uint32_t run = 0;
  for (uint32_t gid = gbeg; gid < gend; gid++, cur ^= 1) {
    cp_async_wait_all();
    __syncthreads();
    if (gid >= img_end) {                                    // the run of tiles of one image ended
      ssim_flush(B, img, run, s_sum);
      run = 0;
      do { img++; img_end = __ldg(B.ss_prefix + img + 1); } while (gid >= img_end);
    }
    uint8_t* ta = cur ? tin1 : tin0;
    uint8_t* tb = ta + SS_INY * SS_PITCH;
    const uint32_t nxt = gid + 1;
    if (nxt < gend) {
      int ni = img;
      while (nxt >= __ldg(B.ss_prefix + ni + 1)) ni++;
      const StatsDesc& nd = B.desc[ni];
      const uint32_t nt = nxt - nd.ss_base;
      uint8_t* na = cur ? tin0 : tin1;
      ssim_stage(nd, (int)(nt % nd.ss_tiles_x) * SS_TX, (int)(nt / nd.ss_tiles_x) * SS_TY, na, na + SS_INY * SS_PITCH);
    }
    cp_async_commit();
    const StatsDesc& d = B.desc[img];
    const uint32_t tile = gid - d.ss_base;
    const int x0 = (int)(tile % d.ss_tiles_x) * SS_TX, y0 = (int)(tile / d.ss_tiles_x) * SS_TY;
    const int H = d.H, W = d.W;

    // horizontal pass: item = (row, 8-column segment)
    for (int item = t; item < SS_HITEMS; item += ST_THREADS) {
      const int r = item >> 3, c0 = (item & 7) * SS_SEG;
      constexpr int NIN = SS_SEG + SS_K - 1;                   // 18 input columns
      float2 v[NIN];                                           // (a - 128, b - 128)
      const uint32_t* wa = reinterpret_cast<const uint32_t*>(ta + r * SS_PITCH + c0);
      const uint32_t* wb = reinterpret_cast<const uint32_t*>(tb + r * SS_PITCH + c0);
#pragma unroll
      for (int w = 0; w < 5; w++) {
        const uint32_t A = wa[w], Bw = wb[w];
#pragma unroll
        for (int k = 0; k < 4; k++) {
          if (w * 4 + k < NIN) {
            const uint32_t sel = (uint32_t)k | 0x7540u;
            const float2 raw = make_float2(__int_as_float((int)__byte_perm(A, 0x4B000000u, sel)),
                                           __int_as_float((int)__byte_perm(Bw, 0x4B000000u, sel)));
            v[w * 4 + k] = make_float2(raw.x + off2.x, raw.y + off2.y);
          }
        }
      }
      float2 o1[SS_SEG];
#pragma unroll
      for (int j = 0; j < SS_SEG; j++) {
        float2 s = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < SS_K; k++) s = fma2(g2[k], v[j + k], s);
        o1[j] = s;
      }
      float4* dst = reinterpret_cast<float4*>(h_ab + r * SS_TX);
#pragma unroll
      for (int j = 0; j < SS_SEG; j += 2)
        dst[swz_chunk((c0 + j) >> 1)] = make_float4(o1[j].x, o1[j].y, o1[j + 1].x, o1[j + 1].y);
      // second pair of planes: (a^2 + b^2, ab); SSIM needs var_a + var_b only as a sum
      float2 q[NIN];
#pragma unroll
      for (int i = 0; i < NIN; i++) q[i] = make_float2(fmaf(v[i].x, v[i].x, v[i].y * v[i].y), v[i].x * v[i].y);
#pragma unroll
      for (int j = 0; j < SS_SEG; j++) {
        float2 s = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < SS_K; k++) s = fma2(g2[k], q[j + k], s);
        o1[j] = s;
      }
      dst = reinterpret_cast<float4*>(h_q + r * SS_TX);
#pragma unroll
      for (int j = 0; j < SS_SEG; j += 2)
        dst[swz_chunk((c0 + j) >> 1)] = make_float4(o1[j].x, o1[j].y, o1[j + 1].x, o1[j + 1].y);
    }
    __syncthreads();

    // vertical pass: thread = (column, 8-row segment)
    const int x = t & (SS_TX - 1), r0 = (t >> 6) * SS_SEG;
    const int xs = 2 * swz_chunk(x >> 1) + (x & 1);          // stored position of column x
    constexpr int NIN = SS_SEG + SS_K - 1;
    float2 mu[SS_SEG], m2[SS_SEG];
    {
      float2 v[NIN];
#pragma unroll
      for (int i = 0; i < NIN; i++) v[i] = h_ab[(r0 + i) * SS_TX + xs];
#pragma unroll
      for (int j = 0; j < SS_SEG; j++) {
        float2 s = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < SS_K; k++) s = fma2(g2[k], v[j + k], s);
        mu[j] = s;
      }
#pragma unroll
      for (int i = 0; i < NIN; i++) v[i] = h_q[(r0 + i) * SS_TX + xs];
#pragma unroll
      for (int j = 0; j < SS_SEG; j++) {
        float2 s = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < SS_K; k++) s = fma2(g2[k], v[j + k], s);
        m2[j] = s;
      }
    }
    const float C1 = (0.01f * 255.f) * (0.01f * 255.f), C2 = (0.03f * 255.f) * (0.03f * 255.f);
    float part = 0.f;
    const bool col_ok = x0 + x <= W - SS_K;
#pragma unroll
    for (int j = 0; j < SS_SEG; j++) {
      const float ma = mu[j].x, mb = mu[j].y;
      // var_a + var_b = E[a^2 + b^2] - mu_a^2 - mu_b^2, cov = E[ab] - mu_a mu_b (centred values)
      const float vsum = m2[j].x - ma * ma - mb * mb, cov = m2[j].y - ma * mb;
      const float ua = ma + 128.f, ub = mb + 128.f;
      const float num = (2.f * ua * ub + C1) * (2.f * cov + C2);
      const float den = (ua * ua + ub * ub + C1) * (vsum + C2);
      // den lies in [C1 C2, 2^33): the fast reciprocal division is accurate to 2 ulp there
      if (col_ok && y0 + r0 + j <= H - SS_K) part += __fdividef(num, den);
    }
    for (int off = 16; off; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
    if ((t & 31) == 0) atomicAdd(&s_sum, (double)part);
    run++;
  }
  __syncthreads();
  ssim_flush(B, img, run, s_sum);
  cp_async_wait_all();
}

}  // namespace rdhei

using namespace rdhei;

namespace {
size_t align256(size_t v) { return (v + 255) / 256 * 256; }

struct StatsLayout {
  size_t desc, chunk_prefix, ss_prefix, total;
  uint32_t chunks, ss_tiles;
};

int stats_layout(const rdhei_stats_job* jobs, int n, StatsLayout& L, std::vector<StatsDesc>* descs) {
  if (n < 0 || (n > 0 && !jobs)) return RDHEI_EINVAL;
  uint64_t chunks = 0, tiles = 0;
  for (int i = 0; i < n; i++) {
    const rdhei_stats_job& j = jobs[i];
    if (j.H < 1 || j.W < 1 || (uint64_t)j.H * j.W > (1ull << 31)) return RDHEI_EINVAL;
    if (!j.a || !j.out || (reinterpret_cast<uintptr_t>(j.out) & 7) || (j.flags & ~RDHEI_STATS_SSIM)) return RDHEI_EINVAL;
    const uint64_t npx = (uint64_t)j.H * j.W;
    const uint32_t nc = (uint32_t)((npx + ST_PX - 1) / ST_PX);
    const bool ss = (j.flags & RDHEI_STATS_SSIM) && j.b && j.H >= SS_K && j.W >= SS_K;
    const uint32_t tx = ss ? (uint32_t)((j.W - SS_K + 1 + SS_TX - 1) / SS_TX) : 0;
    const uint32_t ty = ss ? (uint32_t)((j.H - SS_K + 1 + SS_TY - 1) / SS_TY) : 0;
    if (descs)
      descs->push_back(StatsDesc{j.a, j.b, j.out, npx, j.H, j.W, (uint32_t)chunks, nc, (uint32_t)tiles, tx, tx * ty,
                                 ss ? 1u : 0u});
    chunks += nc;
    tiles += (uint64_t)tx * ty;
  }
  if (chunks >= (1ull << 31) || tiles >= (1ull << 31)) return RDHEI_EINVAL;
  L.chunks = (uint32_t)chunks;
  L.ss_tiles = (uint32_t)tiles;
  L.desc = align256((size_t)n * ST_ACC_WORDS * 4);
  L.chunk_prefix = align256(L.desc + (size_t)n * sizeof(StatsDesc));
  L.ss_prefix = align256(L.chunk_prefix + (size_t)(n + 1) * 4);
  L.total = align256(L.ss_prefix + (size_t)(n + 1) * 4);
  return RDHEI_OK;
}
}  // namespace

extern "C" size_t rdhei_stats_workspace_size(const rdhei_stats_job* jobs, int n) {
  StatsLayout L;
  return stats_layout(jobs, n, L, nullptr) == RDHEI_OK ? L.total : 0;
}

extern "C" size_t rdhei_stats_size(void) { return sizeof(rdhei_stats); }
extern "C" size_t rdhei_stats_job_size(void) { return sizeof(rdhei_stats_job); }

struct rdhei_stats_plan {
  StatsBatch B;
  uint8_t* ws;
  size_t acc_bytes;
  uint32_t chunks, ss_tiles, stats_grid, ssim_grid;
};

extern "C" int rdhei_stats_plan_create(const rdhei_stats_job* jobs, int n, void* ws, size_t ws_bytes, void* stream,
                                       rdhei_stats_plan** out) {
  if (!out) return RDHEI_EINVAL;
  *out = nullptr;
  StatsLayout L;
  std::vector<StatsDesc> descs;
  int rc = stats_layout(jobs, n, L, &descs);
  if (rc) return rc;
  if (n > 0 && (!ws || (reinterpret_cast<uintptr_t>(ws) & 255))) return RDHEI_EINVAL;
  if (n > 0 && ws_bytes < L.total) return RDHEI_ESPACE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  uint8_t* base = static_cast<uint8_t*>(ws);
  if (n > 0) {
    std::vector<uint8_t> host(L.total - L.desc, 0);
    std::memcpy(host.data(), descs.data(), descs.size() * sizeof(StatsDesc));
    uint32_t* cp = reinterpret_cast<uint32_t*>(host.data() + (L.chunk_prefix - L.desc));
    uint32_t* sp = reinterpret_cast<uint32_t*>(host.data() + (L.ss_prefix - L.desc));
    for (int i = 0; i < n; i++) { cp[i] = descs[i].chunk_base; sp[i] = descs[i].ss_base; }
    cp[n] = L.chunks;
    sp[n] = L.ss_tiles;
    if (cudaMemcpyAsync(base + L.desc, host.data(), host.size(), cudaMemcpyHostToDevice, st) != cudaSuccess)
      return RDHEI_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return RDHEI_ECUDA;   // the host copy is released on return
    if (cudaFuncSetAttribute(k_ssim, cudaFuncAttributeMaxDynamicSharedMemorySize, SS_SMEM) != cudaSuccess)
      return RDHEI_ECUDA;
  }
  // k_stats is persistent: as many CTAs as fit on the device at once
  // and so is k_ssim
  int dev = 0, sms = 1, occ = 1, occ_ss = 1;
  if (n > 0 && (cudaGetDevice(&dev) != cudaSuccess ||
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_stats, ST_THREADS, 0) != cudaSuccess ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_ss, k_ssim, ST_THREADS, SS_SMEM) != cudaSuccess))
    return RDHEI_ECUDA;
  rdhei_stats_plan* p = new (std::nothrow) rdhei_stats_plan();
  if (!p) return RDHEI_EINVAL;
  p->ws = base;
  p->acc_bytes = L.desc;
  p->chunks = L.chunks;
  p->ss_tiles = L.ss_tiles;
  p->stats_grid = std::min<uint32_t>(L.chunks, (uint32_t)std::max(1, sms * std::max(occ, 1)));
  p->ssim_grid = std::min<uint32_t>(L.ss_tiles, (uint32_t)std::max(1, sms * std::max(occ_ss, 1)));
  StatsBatch& B = p->B;
  B.desc = reinterpret_cast<const StatsDesc*>(base + L.desc);
  B.chunk_prefix = reinterpret_cast<const uint32_t*>(base + L.chunk_prefix);
  B.ss_prefix = reinterpret_cast<const uint32_t*>(base + L.ss_prefix);
  B.n = n;
  B.total_chunks = L.chunks;
  B.total_ss_tiles = L.ss_tiles;
  B.acc = reinterpret_cast<uint32_t*>(base);
  double g[SS_K], gs = 0.0;
  for (int k = 0; k < SS_K; k++) {
    const double u = k - (SS_K - 1) / 2;
    g[k] = std::exp(-u * u / (2.0 * 1.5 * 1.5));
    gs += g[k];
  }
  for (int k = 0; k < SS_K; k++) B.g[k] = (float)(g[k] / gs);
  *out = p;
  return RDHEI_OK;
}

extern "C" int rdhei_stats_plan_run_stage(rdhei_stats_plan* p, int stage, void* stream) {
  if (!p || stage < 0 || stage > 1) return RDHEI_EINVAL;
  if (p->B.n == 0) return RDHEI_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (stage == 0) {
    if (cudaMemsetAsync(p->ws, 0, p->acc_bytes, st) != cudaSuccess) return RDHEI_ECUDA;
    k_stats<<<p->stats_grid, ST_THREADS, 0, st>>>(p->B);
  } else if (p->ss_tiles) {
    k_ssim<<<p->ssim_grid, ST_THREADS, SS_SMEM, st>>>(p->B);
  }
  return cudaGetLastError() == cudaSuccess ? RDHEI_OK : RDHEI_ECUDA;
}

extern "C" int rdhei_stats_plan_run(rdhei_stats_plan* p, void* stream) {
  NvtxRange range("rdhei_image_stats");
  int rc = rdhei_stats_plan_run_stage(p, 0, stream);
  return rc ? rc : rdhei_stats_plan_run_stage(p, 1, stream);
}

extern "C" void rdhei_stats_plan_destroy(rdhei_stats_plan* p) { delete p; }

extern "C" int rdhei_image_stats(const rdhei_stats_job* jobs, int n, void* ws, size_t ws_bytes, void* stream) {
  rdhei_stats_plan* p = nullptr;
  int rc = rdhei_stats_plan_create(jobs, n, ws, ws_bytes, stream, &p);
  if (rc) return rc;
  rc = rdhei_stats_plan_run(p, stream);
  rdhei_stats_plan_destroy(p);
  return rc;
}
