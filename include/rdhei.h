/*
 * rdhei.h -- C ABI of the GB300 (sm_103a) implementation of multi-MSB replacement
 * reversible data hiding in encrypted images (EMR-RDHEI and the per-pixel stages of
 * LMR-RDHEI; Zhang & Luo, "Vector-based Efficient Data Hiding in Encrypted Images via
 * Multi-MSB Replacement", arXiv 2302.07992).
 *
 * Four calls follow the paper's three parties (Fig. General_EMR, Fig. General_LMR):
 *   content owner  rdhei_label_encrypt    Sec. III-A-1 / III-B-1
 *   data hider     rdhei_embed            Sec. III-A-2 / III-B-2
 *   receiver (K2)  rdhei_extract          Sec. III-A-3 / III-B-3, "receiver has only K2"
 *   receiver (K1)  rdhei_decrypt_recover  Sec. III-A-3 / III-B-3, "receiver has only K1"
 * Each works on a batch of images of any sizes (one image is a batch of one).
 *
 * Conventions shared by every call
 * --------------------------------
 * Images: 8-bit grayscale, H rows x W columns, row-major, no padding, in DEVICE memory.
 *   1 <= H, W <= 65536 and H * W <= 2^27.
 * Bit streams (payload, extracted bits, packed location map l, packed first-MSB map
 *   eta, LMR side bits): bit k is bit (7 - k % 8) of byte k / 8 (most significant bit
 *   first).  Device buffers holding a stream of n bits must be 4-byte aligned and
 *   readable/writable up to ceil(n / 32) * 4 bytes.
 * Packed maps are in raster order of the ROTATED (encrypted) domain: bit q is pixel q.
 * Keystreams: ChaCha20 (RFC 8439) with a 256-bit key, 96-bit nonce and block counter
 *   from 0.  s(i, j) = byte i * W + j of the K1 stream (Sec. "Secret key generation":
 *   "reshaped into the input image's size"); the hider's stream z2 is the K2 stream read
 *   as bits in the stream convention above, and payload bit k is sent as m(k) XOR z2(k).
 * Rotation: levels L = lmin .. n, n = floor(log2(min(H, W))); each aligned 2^L x 2^L
 *   block that lies inside the image is turned counter-clockwise by a quarter-turns,
 *   a = (sum of s over the block) mod 4 (Eq. roration); decoding runs the levels in
 *   reverse with (4 - a) mod 4 (Eq. roration2).  lmin = 0 selects the default: 1 for
 *   EMR, 4 for LMR (the 2^4 .. 2^9 blocks the paper uses at 512 x 512), clamped to n.
 * Payload slots: label-0 pixels in raster order of the rotated domain; each gives b
 *   (EMR) or b - 1 (LMR) slots, filled from bit 7 (EMR) or bit 6 (LMR) downwards.
 * Streams and memory: every call is asynchronous on the caller's CUDA stream
 *   (passed as void*, a cudaStream_t).  The library never allocates device memory:
 *   the caller passes a workspace of rdhei_workspace_size() bytes (256-byte aligned).
 *   Calls that share a workspace must be ordered on one stream.
 * Errors: calls return an rdhei_status code for argument errors found on the host.
 *   Errors that only the device can see (payload longer than the capacity, a
 *   look-back wait that timed out) are written to the per-image rdhei_info.status
 *   and to a workspace-wide word read by rdhei_workspace_status().
 */
#ifndef RDHEI_H
#define RDHEI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum rdhei_status {
    RDHEI_OK = 0,
    RDHEI_EINVAL = 1,     /* bad size, b, variant, null pointer or misaligned buffer */
    RDHEI_ECAPACITY = 2,  /* payload longer than the capacity: only the capacity is embedded */
    RDHEI_ECUDA = 3,      /* a CUDA runtime call failed */
    RDHEI_ETIMEOUT = 4,   /* a bounded device-side wait gave up; outputs are invalid */
    RDHEI_ESPACE = 5      /* workspace too small */
};

enum rdhei_variant { RDHEI_EMR = 0, RDHEI_LMR = 1 };

/* Per-image results, written by the device into caller-owned device memory. */
typedef struct rdhei_info {
    uint32_t hist[9];     /* label histogram: hist[t] = #pixels sharing exactly t leading
                             bits with their left neighbour (t = 8: equal; first column: t = 0);
                             zeros(b) = sum_{t >= b} hist[t] is the b-MSB map's label-0 count */
    int32_t  b;           /* b used by label_encrypt (Eq. optimal_b when requested) */
    uint64_t capacity;    /* payload capacity in bits: b * zeros(b) (EMR), (b-1) * zeros(b) (LMR) */
    uint64_t embedded;    /* bits written by rdhei_embed = min(nbits, capacity) */
    uint64_t extracted;   /* bits written by rdhei_extract = min(max_bits, capacity) */
    int32_t  status;      /* rdhei_status of the last device-side step for this image */
    int32_t  reserved;
} rdhei_info;

/* One image of a batch.  Pointers are device pointers; unused ones may be NULL. */
typedef struct rdhei_job {
    int32_t H, W;
    int32_t variant;      /* RDHEI_EMR or RDHEI_LMR */
    int32_t b;            /* label_encrypt: 0 = choose by Eq. optimal_b (EMR b in [2,7],
                             LMR b in [2,8], ties to the smaller b), else fixed.
                             embed / extract / decrypt_recover: the public b; 0 = read
                             info->b as written by an earlier label_encrypt. */
    int32_t rot_lmin;     /* 0 = default (see above) */
    int32_t rot_enable;   /* 0 = no rotation (all angles 0) */
    uint8_t k1[32], nonce1[12];   /* image key K1 (content owner, K1 receiver) */
    uint8_t k2[32], nonce2[12];   /* data hiding key K2 (hider, K2 receiver) */
    const uint8_t *src;   /* label_encrypt: I; embed: I_e; extract, decrypt_recover: I_e' */
    uint8_t *dst;         /* label_encrypt: I_e; embed: I_e' (may equal src); decrypt_recover: I' */
    uint8_t *map_bits;    /* label_encrypt: out, rotated l (optional for EMR, whose map is the
                             LSB plane); LMR embed / extract / decrypt_recover: in */
    uint8_t *eta_bits;    /* label_encrypt: out, rotated eta (LMR, optional);
                             LMR decrypt_recover: in */
    const uint8_t *side_bits;  /* LMR label_encrypt: the compressed maps written into bit 7
                                  of the first side_nbits pixels; NULL keeps the ciphertext */
    uint64_t side_nbits;
    const uint8_t *payload;    /* embed: message bits (before K2 encryption) */
    uint64_t nbits;            /* embed: message length in bits */
    uint8_t *bits_out;         /* extract: decrypted message bits */
    uint64_t max_bits;         /* extract: at most this many bits are written */
    rdhei_info *info;          /* device, required */
} rdhei_job;

/* Workspace bytes needed for this batch (host-only computation). */
size_t rdhei_workspace_size(const rdhei_job *jobs, int n);

/* Content owner (Sec. III-A-1, III-B-1): label histogram and b (Eqs. gliding1/2,
 * optimal_b), location map l and first-MSB map eta (Eq. MSB_map), key-driven block
 * rotation (Eq. roration), XOR encryption (Eq. image_encryption), and the map
 * embedding: EMR writes rotated l into the LSB plane; LMR writes side_bits into bit 7.
 * Writes job.dst, job.map_bits / eta_bits (if given) and info->{hist, b, capacity}. */
int rdhei_label_encrypt(const rdhei_job *jobs, int n, void *ws, size_t ws_bytes, void *stream);

/* Data hider (Sec. III-A-2, III-B-2): encrypts the payload with z2 and writes it into
 * the b (EMR) or b-1 (LMR) slots of label-0 pixels, read from the LSB plane (EMR) or
 * from job.map_bits (LMR).  Writes job.dst and info->embedded; if nbits exceeds the
 * capacity the first `capacity` bits are embedded and info->status = RDHEI_ECAPACITY. */
int rdhei_embed(const rdhei_job *jobs, int n, void *ws, size_t ws_bytes, void *stream);

/* Receiver with K2 (Sec. III-A-3, III-B-3): concatenates the slots of label-0 pixels
 * (no de-rotation) and decrypts with z2.  Writes min(max_bits, capacity) bits to
 * job.bits_out, zero-filling the last partial 32-bit word, and info->extracted. */
int rdhei_extract(const rdhei_job *jobs, int n, void *ws, size_t ws_bytes, void *stream);

/* Receiver with K1 (Sec. III-A-3, III-B-3, Eq. roration2): XOR decryption, de-rotation,
 * and row-wise restoration of the replaced MSBs from the last label-1 pixel to the
 * left.  EMR: the map is the LSB plane and the output LSB is the decrypted LSB.  LMR:
 * job.map_bits and job.eta_bits (decompressed side information) are inputs; bit 7 comes
 * from eta and the result is lossless.  Writes job.dst. */
int rdhei_decrypt_recover(const rdhei_job *jobs, int n, void *ws, size_t ws_bytes, void *stream);

/* LMR side information into bit 7 of an encrypted image (Sec. III-B-1, "Maps
 * embedding"): pixel q < side_nbits gets bit 7 := side bit q.  In place on job.dst. */
int rdhei_lmr_set_side(const rdhei_job *jobs, int n, void *ws, size_t ws_bytes, void *stream);

/* ---------------------------------------------------------------------------------
 * Plans: the calls above re-validate, re-lay-out and re-upload the batch's
 * descriptors on every call (a host-synchronous copy).  A plan does that once:
 *   rdhei_plan_create  validates the jobs and computes the workspace layout (host only);
 *   rdhei_plan_upload  writes the descriptors into the workspace (host-synchronous;
 *                      not allowed during stream capture);
 *   rdhei_plan_run     launches one operation (memsets and kernels only, so it can be
 *                      captured into a CUDA graph and replayed);
 *   rdhei_plan_destroy frees the host-side object.
 * The jobs' pointers are baked into the plan: to use new buffers, make a new plan.
 * ------------------------------------------------------------------------------- */
enum rdhei_op {
    RDHEI_OP_LABEL_ENCRYPT = 0,
    RDHEI_OP_EMBED = 1,
    RDHEI_OP_EXTRACT = 2,
    RDHEI_OP_DECRYPT_RECOVER = 3,
    RDHEI_OP_LMR_SET_SIDE = 4
};
typedef struct rdhei_plan rdhei_plan;
int rdhei_plan_create(const rdhei_job *jobs, int n, rdhei_plan **plan);
size_t rdhei_plan_workspace_size(const rdhei_plan *plan);
int rdhei_plan_upload(rdhei_plan *plan, void *ws, size_t ws_bytes, void *stream);
int rdhei_plan_run(rdhei_plan *plan, int op, void *stream);
void rdhei_plan_destroy(rdhei_plan *plan);

/* The kernels of one operation, one launch per stage, for timing each kernel with
 * events recorded between stages: stage 0 also issues the per-call workspace memsets.
 * rdhei_plan_run(plan, op) == every stage of op in order.  Unknown op: 0 stages. */
int rdhei_plan_stage_count(int op);
const char *rdhei_stage_name(int op, int stage);
int rdhei_plan_run_stage(rdhei_plan *plan, int op, int stage, void *stream);

/* ---------------------------------------------------------------------------------
 * Extraction without any allocation.  The paper has no counterpart to this call; it
 * exists for callers that cannot allocate device memory at all -- code that runs in a
 * host callback or under a runtime that owns every allocation, or a tool that links
 * only this library -- and so cannot hand rdhei_extract a workspace.  It does what
 * rdhei_extract does for ONE image (job->src, job->map_bits for LMR, job->bits_out,
 * job->max_bits, job->info, job->b, K2) with the kernels rdhei_extract uses, and
 * calls no cudaMalloc, cudaFree or other allocating routine.
 *   Scratch: a file-scope device array of about 17 KB that the CUDA runtime sets up
 *     when the library loads; every GPU that loads the library holds it until exit.
 *   Limit: H * W <= RDHEI_NOALLOC_MAX_PIXELS (2^24); larger images return
 *     RDHEI_ESPACE before any GPU work.
 *   First call on a device: looks the array's device address up (cudaGetSymbolAddress
 *     with that device current) and caches it; make it before any stream capture.
 *   Sharing: every call uses the same array and it keeps the last call's contents;
 *     what must start at zero is cleared on each call.  Calls whose work overlaps on
 *     the GPU (other streams, other threads) race: order them on one stream.
 *   Returns RDHEI_EINVAL for bad arguments, RDHEI_ECUDA for a failed CUDA call. */
#define RDHEI_NOALLOC_MAX_PIXELS (1u << 24)
int rdhei_extract_noalloc(const rdhei_job *job, void *stream);

/* Workspace-wide device error word of the most recent call on this workspace
 * (synchronises the stream).  0 = no error, else an rdhei_status code. */
int rdhei_workspace_status(void *ws, void *stream, int32_t *code);

/* sizeof(rdhei_job) and sizeof(rdhei_info), for bindings that build them by hand. */
size_t rdhei_job_size(void);
size_t rdhei_info_size(void);

/* Library version and build target, e.g. "rdhei 0.1 sm_103a". */
const char *rdhei_version(void);

#ifdef __cplusplus
}
#endif
#endif /* RDHEI_H */
