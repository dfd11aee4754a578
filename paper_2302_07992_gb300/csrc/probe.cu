// probe.cu -- measured ceilings of the integer work on this GPU, for the roofline of
// the path's kernels (which are bound by the integer/logic pipe, not by HBM):
//   k_probe_alu        the integer/logic (ALU) pipe alone: independent chains of
//                      three-input XORs and funnel-shift rotations -- the two operation
//                      kinds of ChaCha20's quarter-round that do not go to the FMA pipe;
//   k_probe_keystream  the ChaCha20 keystream alone, with the block function the path's
//                      kernels use (chacha20_block<2>), XOR-folded into one word per
//                      thread so that nothing but the cipher is timed.
#include "../../include/rdhei.h"
#include "common.cuh"

namespace rdhei {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_CHAINS = 8;   // independent dependency chains per thread

// Each iteration issues, per chain, one XOR with a per-chain constant (LOP3) and one
// rotation (SHF): 2 * PROBE_CHAINS ALU-pipe operations per thread and iteration; the
// loop counter's own instructions are amortised over four unrolled iterations.
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_alu(uint32_t* out, int iters, uint32_t seed) {
  uint32_t v[PROBE_CHAINS], kc[PROBE_CHAINS];
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; c++) {
    v[c] = seed * (threadIdx.x + 1) + 0x9E3779B9u * (c + 1) + blockIdx.x;
    kc[c] = (seed ^ blockIdx.x) + 0x6D2B79F5u * (uint32_t)c;
  }
#pragma unroll 4
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; c++) v[c] = __funnelshift_l(v[c] ^ kc[c], v[c] ^ kc[c], 7 + c);
  }
  uint32_t r = 0;
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; c++) r ^= v[c];
  out[blockIdx.x * PROBE_THREADS + threadIdx.x] = r;
}

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_keystream(uint32_t* out, int per_thread, Batch B) {
  const ImgDesc& d = B.desc[0];
  const uint32_t g = blockIdx.x * PROBE_THREADS + threadIdx.x;
  uint32_t acc = 0;
  for (int i = 0; i < per_thread; i++) {
    uint32_t o[16];
    chacha20_block<2>(d.k1, g * (uint32_t)per_thread + (uint32_t)i, d.n1, o, d.one);
#pragma unroll
    for (int k = 0; k < 16; k++) acc ^= o[k];
  }
  out[g] = acc;
}

}  // namespace rdhei

using namespace rdhei;

extern "C" {

int rdhei_probe_alu(uint32_t* out, int blocks, int iters, void* stream) {
  if (!out || blocks < 1 || iters < 1 || (reinterpret_cast<uintptr_t>(out) & 3)) return RDHEI_EINVAL;
  k_probe_alu<<<blocks, PROBE_THREADS, 0, reinterpret_cast<cudaStream_t>(stream)>>>(out, iters, 0x2545F491u);
  return cudaGetLastError() == cudaSuccess ? RDHEI_OK : RDHEI_ECUDA;
}

int rdhei_probe_keystream(uint32_t* out, int blocks, int per_thread, const rdhei_job* key_job, void* ws,
                          void* stream) {
  if (!out || !key_job || !ws || blocks < 1 || per_thread < 1) return RDHEI_EINVAL;
  if ((reinterpret_cast<uintptr_t>(out) & 3) || (reinterpret_cast<uintptr_t>(ws) & 15)) return RDHEI_EINVAL;
  // one descriptor (K1, nonce1) in the caller's workspace
  ImgDesc d = {};
  for (int k = 0; k < 8; k++)
    d.k1[k] = (uint32_t)key_job->k1[4 * k] | ((uint32_t)key_job->k1[4 * k + 1] << 8) |
              ((uint32_t)key_job->k1[4 * k + 2] << 16) | ((uint32_t)key_job->k1[4 * k + 3] << 24);
  for (int k = 0; k < 3; k++)
    d.n1[k] = (uint32_t)key_job->nonce1[4 * k] | ((uint32_t)key_job->nonce1[4 * k + 1] << 8) |
              ((uint32_t)key_job->nonce1[4 * k + 2] << 16) | ((uint32_t)key_job->nonce1[4 * k + 3] << 24);
  d.one = 1;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(ws, &d, sizeof(d), cudaMemcpyHostToDevice, st) != cudaSuccess) return RDHEI_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return RDHEI_ECUDA;   // d leaves scope
  Batch B = {};
  B.desc = reinterpret_cast<const ImgDesc*>(ws);
  k_probe_keystream<<<blocks, PROBE_THREADS, 0, st>>>(out, per_thread, B);
  return cudaGetLastError() == cudaSuccess ? RDHEI_OK : RDHEI_ECUDA;
}

size_t rdhei_probe_workspace_size(void) { return sizeof(ImgDesc); }

}  // extern "C"
