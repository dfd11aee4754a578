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
// runs the horizontal 11-tap pass over all 42 rows into five shared planes (mu_a, mu_b,
// E[a^2], E[b^2], E[ab], pixels centred at 128), then the vertical pass with eight
// outputs per thread, combines the local moments into the SSIM of each window and
// adds the window sum into the image's fp64 accumulator.  The last CTA of an image
// writes the mean.
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
constexpr int SS_PITCH = 76;             // bytes per staged input row (word multiple)
constexpr int SS_SEG = 8;                // horizontal outputs per item, vertical outputs per thread
constexpr int SS_HITEMS = SS_INY * (SS_TX / SS_SEG);   // 336 horizontal items
constexpr int SS_SMEM = 2 * SS_INY * SS_PITCH + 5 * SS_INY * SS_TX * 4;   // 60144 bytes

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
  uint32_t* acc;                       // n * ST_ACC_WORDS, zeroed per call
  float g[SS_K];                       // normalised 1-D Gaussian, sigma 1.5
};

__device__ __forceinline__ float centred(uint32_t word, int k) {
  // byte k of word as a float minus 128: 2^23 + byte assembled by one byte permute
  const uint32_t sel = (uint32_t)k | 0x7540u;
  return __int_as_float((int)__byte_perm(word, 0x4B000000u, sel)) - 8388736.0f;
}

__global__ void __launch_bounds__(ST_THREADS) k_stats(StatsBatch B) {
  __shared__ uint32_t h[ST_THREADS / 32][256];
  __shared__ unsigned long long s_abs, s_sq;
  __shared__ uint32_t s_diff, s_last;
  const int t = threadIdx.x, warp = t >> 5;
  const uint32_t g = blockIdx.x;
  const int img = owner_of(B.chunk_prefix, B.n, g);
  const StatsDesc& d = B.desc[img];
  for (int i = t; i < (ST_THREADS / 32) * 256; i += ST_THREADS) (&h[0][0])[i] = 0u;
  if (t == 0) { s_abs = 0; s_sq = 0; s_diff = 0; }
  __syncthreads();

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
    for (int k = 0; k < 32; k++) {
      if (k < valid) {
        const uint32_t x = (wa[k >> 2] >> (8 * (k & 3))) & 0xFFu;
        atomicAdd(&h[warp][x], 1u);
        if (pb) {
          const uint32_t y = (wb[k >> 2] >> (8 * (k & 3))) & 0xFFu;
          const uint32_t ad = x > y ? x - y : y - x;
          ndiff += ad != 0;
          sabs += ad;
          ssq += ad * ad;
        }
      }
    }
  }
  // warp sums fit 32 bits: at most 32 lanes x 32 pixels x 255^2
  ndiff = __reduce_add_sync(0xffffffffu, ndiff);
  sabs = __reduce_add_sync(0xffffffffu, sabs);
  ssq = __reduce_add_sync(0xffffffffu, ssq);
  if ((t & 31) == 0) {
    atomicAdd(&s_diff, ndiff);
    atomicAdd(&s_abs, (unsigned long long)sabs);
    atomicAdd(&s_sq, (unsigned long long)ssq);
  }
  __syncthreads();
  uint32_t* acc = B.acc + (size_t)img * ST_ACC_WORDS;
  for (int v = t; v < 256; v += ST_THREADS) {
    uint32_t c = 0;
#pragma unroll
    for (int w = 0; w < ST_THREADS / 32; w++) c += h[w][v];
    if (c) atomicAdd(acc + v, c);
  }
  __syncthreads();
  if (t == 0) {
    atomicAdd(acc + ACC_NDIFF, s_diff);
    atomicAdd(reinterpret_cast<unsigned long long*>(acc + ACC_ABS), s_abs);
    atomicAdd(reinterpret_cast<unsigned long long*>(acc + ACC_SQ), s_sq);
    __threadfence();
    s_last = atomicAdd(acc + ACC_DONE, 1u) + 1 == d.nchunks;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // last CTA of the image: the metrics in fp64
  rdhei_stats* out = d.out;
  for (int v = t; v < 256; v += ST_THREADS) out->hist[v] = __ldcg(acc + v);
  if (t == 0) {
    const double N = (double)d.npx;
    double H = 0.0, chi = 0.0;
    for (int v = 0; v < 256; v++) {
      const uint32_t c = __ldcg(acc + v);
      const double P = (double)c / N;
      if (c) H -= P * log2(P);
      chi += (P - 1.0 / 256.0) * (P - 1.0 / 256.0);
    }
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
}

__global__ void __launch_bounds__(ST_THREADS, 3) k_ssim(StatsBatch B) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint8_t* ta = smem;                                        // [SS_INY][SS_PITCH]
  uint8_t* tb = smem + SS_INY * SS_PITCH;
  float* hs = reinterpret_cast<float*>(smem + 2 * SS_INY * SS_PITCH);   // [5][SS_INY][SS_TX]
  __shared__ double s_sum;
  __shared__ uint32_t s_last;
  const int t = threadIdx.x;
  const uint32_t gid = blockIdx.x;
  const int img = owner_of(B.ss_prefix, B.n, gid);
  const StatsDesc& d = B.desc[img];
  const uint32_t tile = gid - d.ss_base;
  const int x0 = (int)(tile % d.ss_tiles_x) * SS_TX, y0 = (int)(tile / d.ss_tiles_x) * SS_TY;
  const int H = d.H, W = d.W;
  if (t == 0) s_sum = 0.0;

  // stage the input rectangle of both images; zeros outside the image feed only
  // window positions that are masked out below
  const bool words = (W & 3) == 0 && ((reinterpret_cast<uintptr_t>(d.a) | reinterpret_cast<uintptr_t>(d.b)) & 3) == 0;
  if (words) {
    constexpr int WPR = SS_PITCH / 4;                        // 19 words per staged row
    for (int i = t; i < SS_INY * WPR; i += ST_THREADS) {
      const int r = i / WPR, c = (i - r * WPR) * 4;
      const int y = y0 + r, x = x0 + c;
      uint32_t va = 0, vb = 0;
      if (y < H && x < W) {
        const size_t o = (size_t)y * W + x;
        va = __ldg(reinterpret_cast<const uint32_t*>(d.a + o));
        vb = __ldg(reinterpret_cast<const uint32_t*>(d.b + o));
      }
      *reinterpret_cast<uint32_t*>(ta + r * SS_PITCH + c) = va;
      *reinterpret_cast<uint32_t*>(tb + r * SS_PITCH + c) = vb;
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
  __syncthreads();

  // horizontal pass: item = (row, 8-column segment) -> five planes of 8 outputs
  for (int item = t; item < SS_HITEMS; item += ST_THREADS) {
    const int r = item >> 3, c0 = (item & 7) * SS_SEG;
    float pa[SS_SEG + SS_K - 1], pb[SS_SEG + SS_K - 1];      // 18 centred pixels each
    const uint32_t* wa = reinterpret_cast<const uint32_t*>(ta + r * SS_PITCH + c0);
    const uint32_t* wb = reinterpret_cast<const uint32_t*>(tb + r * SS_PITCH + c0);
#pragma unroll
    for (int w = 0; w < 5; w++) {
      const uint32_t A = wa[w], Bw = wb[w];
#pragma unroll
      for (int k = 0; k < 4; k++) {
        if (w * 4 + k < SS_SEG + SS_K - 1) {
          pa[w * 4 + k] = centred(A, k);
          pb[w * 4 + k] = centred(Bw, k);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 5; q++) {
      float v[SS_SEG + SS_K - 1];
#pragma unroll
      for (int i = 0; i < SS_SEG + SS_K - 1; i++)
        v[i] = q == 0 ? pa[i] : q == 1 ? pb[i] : q == 2 ? pa[i] * pa[i] : q == 3 ? pb[i] * pb[i] : pa[i] * pb[i];
      float o[SS_SEG];
#pragma unroll
      for (int j = 0; j < SS_SEG; j++) {
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < SS_K; k++) s = fmaf(B.g[k], v[j + k], s);
        o[j] = s;
      }
      float4* dst = reinterpret_cast<float4*>(hs + (q * SS_INY + r) * SS_TX + c0);
      dst[0] = make_float4(o[0], o[1], o[2], o[3]);
      dst[1] = make_float4(o[4], o[5], o[6], o[7]);
    }
  }
  __syncthreads();

  // vertical pass: thread = (column, 8-row segment)
  const int x = t & (SS_TX - 1), r0 = (t >> 6) * SS_SEG;
  float m[5][SS_SEG];
#pragma unroll
  for (int q = 0; q < 5; q++) {
    float v[SS_SEG + SS_K - 1];
#pragma unroll
    for (int i = 0; i < SS_SEG + SS_K - 1; i++) v[i] = hs[(q * SS_INY + r0 + i) * SS_TX + x];
#pragma unroll
    for (int j = 0; j < SS_SEG; j++) {
      float s = 0.f;
#pragma unroll
      for (int k = 0; k < SS_K; k++) s = fmaf(B.g[k], v[j + k], s);
      m[q][j] = s;
    }
  }
  const float C1 = (0.01f * 255.f) * (0.01f * 255.f), C2 = (0.03f * 255.f) * (0.03f * 255.f);
  float part = 0.f;
  const bool col_ok = x0 + x <= W - SS_K;
#pragma unroll
  for (int j = 0; j < SS_SEG; j++) {
    const float ma = m[0][j], mb = m[1][j];
    const float va = m[2][j] - ma * ma, vb = m[3][j] - mb * mb, cov = m[4][j] - ma * mb;
    const float ua = ma + 128.f, ub = mb + 128.f;
    const float num = (2.f * ua * ub + C1) * (2.f * cov + C2);
    const float den = (ua * ua + ub * ub + C1) * (va + vb + C2);
    if (col_ok && y0 + r0 + j <= H - SS_K) part += num / den;
  }
  for (int off = 16; off; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
  if ((t & 31) == 0) atomicAdd(&s_sum, (double)part);
  __syncthreads();
  uint32_t* acc = B.acc + (size_t)img * ST_ACC_WORDS;
  if (t == 0) {
    atomicAdd(reinterpret_cast<double*>(acc + ACC_SSIM), s_sum);
    __threadfence();
    s_last = atomicAdd(acc + ACC_SSIM_DONE, 1u) + 1 == d.ss_ntiles;
  }
  __syncthreads();
  if (t == 0 && s_last) {
    __threadfence();
    const double sum = __ldcg(reinterpret_cast<const double*>(acc + ACC_SSIM));
    d.out->ssim = sum / ((double)(H - SS_K + 1) * (double)(W - SS_K + 1));
  }
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
  uint32_t chunks, ss_tiles;
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
  rdhei_stats_plan* p = new (std::nothrow) rdhei_stats_plan();
  if (!p) return RDHEI_EINVAL;
  p->ws = base;
  p->acc_bytes = L.desc;
  p->chunks = L.chunks;
  p->ss_tiles = L.ss_tiles;
  StatsBatch& B = p->B;
  B.desc = reinterpret_cast<const StatsDesc*>(base + L.desc);
  B.chunk_prefix = reinterpret_cast<const uint32_t*>(base + L.chunk_prefix);
  B.ss_prefix = reinterpret_cast<const uint32_t*>(base + L.ss_prefix);
  B.n = n;
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
    k_stats<<<p->chunks, ST_THREADS, 0, st>>>(p->B);
  } else if (p->ss_tiles) {
    k_ssim<<<p->ss_tiles, ST_THREADS, SS_SMEM, st>>>(p->B);
  }
  return cudaGetLastError() == cudaSuccess ? RDHEI_OK : RDHEI_ECUDA;
}

extern "C" int rdhei_stats_plan_run(rdhei_stats_plan* p, void* stream) {
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
