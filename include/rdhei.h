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
 * Two fused calls run two parties back to back with fewer passes over memory:
 *   owner + hider  rdhei_encode           Sec. III-A-1 then III-A-2 (III-B-1, III-B-2)
 *   both keys      rdhei_decode           Sec. III-A-3 / III-B-3, "receiver has both keys"
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
    RDHEI_ESPACE = 5,     /* workspace too small */
    RDHEI_EBOUNDS = 6     /* checked build (-DRDHEI_CHECK) only: a device index check failed
                             and the access was skipped; outputs are invalid */
};

/* RDHEI_EMR / RDHEI_LMR are the paper's methods: labels compare a pixel's top b bits
 * with the left neighbour's (the glide of Eqs. gliding1/2).  RDHEI_EMR_MED /
 * RDHEI_LMR_MED are a RELATED-WORK variant, not the paper's method: labels compare
 * with the median edge detector (MED, LOCO-I) prediction that Sec. II quotes from
 * Puyang et al. and Puteaux et al.,
 *   pred = min(A, B) if C >= max(A, B); max(A, B) if C <= min(A, B); A + B - C else,
 * A, B, C the left, upper and upper-left neighbours (row 0 predicts from the left,
 * column 0 from above, pixel (0, 0) is never redundant; the EMR form predicts on the
 * top seven bits, since the receiver loses the LSB plane).  Everything else (b,
 * rotation, encryption, hiding) is as in the base variant.  Recovery then depends on
 * the recovered left, upper and upper-left pixels, so rdhei_decrypt_recover runs it
 * as a tiled anti-diagonal wavefront (plan stage 3). */
enum rdhei_variant { RDHEI_EMR = 0, RDHEI_LMR = 1, RDHEI_EMR_MED = 2, RDHEI_LMR_MED = 3 };

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
    int32_t variant;      /* enum rdhei_variant */
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

/* Owner and hider in one call (Sec. III-A-1 followed by Sec. III-A-2; Sec. III-B-1
 * followed by Sec. III-B-2): the result equals rdhei_label_encrypt followed by
 * rdhei_embed with the b it chose, bit for bit, in three kernels instead of eight.  The
 * payload slots of each 64-row strip of the rotated image start at a bit offset derived
 * from per-tile label counts of the first pass, so each strip is encrypted and then
 * filled with the K2-encrypted payload by one CTA while it is still in L2.
 * Job fields: src = I, dst = I_e' (the marked image; must not alias src), payload /
 * nbits, K1 and K2; LMR: map_bits is REQUIRED (the rotated map is written there and
 * read back by the hider's half), eta_bits optional, side_bits / side_nbits as for
 * rdhei_label_encrypt (the compressed maps must therefore be known before the call; an
 * owner that compresses the maps it is computing uses the separable calls).
 * Writes dst, map_bits / eta_bits, info->{hist, b, capacity, embedded}; a payload longer
 * than the capacity embeds the capacity and sets info->status = RDHEI_ECAPACITY. */
int rdhei_encode(const rdhei_job *jobs, int n, void *ws, size_t ws_bytes, void *stream);

/* Receiver with both keys (Sec. III-A-3 / III-B-3, "the receiver has both keys"): the
 * result equals rdhei_extract followed by rdhei_decrypt_recover, bit for bit.  The first
 * pass (K1 keystream, decryption, rotation angles) also counts each tile's payload
 * slots, so the extraction kernel starts every 64-row strip at its bit offset and
 * decrypts with K2 as it writes -- no count pass and no separate K2 pass.
 * Job fields: src = I_e', dst = I' (must not alias src), bits_out / max_bits, b (0 =
 * info->b), K1 and K2; LMR: map_bits and eta_bits required.  Writes bits_out
 * (min(max_bits, capacity) bits, the last partial word zero-filled), dst and
 * info->extracted. */
int rdhei_decode(const rdhei_job *jobs, int n, void *ws, size_t ws_bytes, void *stream);

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
    RDHEI_OP_LMR_SET_SIDE = 4,
    RDHEI_OP_ENCODE = 5,
    RDHEI_OP_DECODE = 6
};
typedef struct rdhei_plan rdhei_plan;
int rdhei_plan_create(const rdhei_job *jobs, int n, rdhei_plan **plan);
size_t rdhei_plan_workspace_size(const rdhei_plan *plan);
int rdhei_plan_upload(rdhei_plan *plan, void *ws, size_t ws_bytes, void *stream);
/* The same without waiting: the descriptors are written into `staging` (caller-owned
 * PAGE-LOCKED host memory of at least rdhei_plan_staging_size() bytes) and copied from
 * there asynchronously on `stream`; the caller keeps `staging` untouched until the
 * stream has passed the copy (for example until the plan's work on that stream has
 * completed).  Returns RDHEI_ESPACE for a staging buffer that is too small. */
size_t rdhei_plan_staging_size(const rdhei_plan *plan);
int rdhei_plan_upload_async(rdhei_plan *plan, void *ws, size_t ws_bytes, void *staging, size_t staging_bytes,
                            void *stream);
int rdhei_plan_run(rdhei_plan *plan, int op, void *stream);
void rdhei_plan_destroy(rdhei_plan *plan);

/* The kernels of one operation, one launch per stage, for timing each kernel with
 * events recorded between stages: stage 0 also clears the per-call region of the
 * workspace (one kernel, or a memset when that region is not 16-byte aligned).
 * rdhei_plan_run(plan, op) == every stage of op in order.  Unknown op: 0 stages.
 * rdhei_plan_stage_active: 1 when the stage launches work for this plan's jobs (the
 * MED wavefront stage of rdhei_decrypt_recover launches only for MED variants). */
int rdhei_plan_stage_count(int op);
const char *rdhei_stage_name(int op, int stage);
int rdhei_plan_run_stage(rdhei_plan *plan, int op, int stage, void *stream);
int rdhei_plan_stage_active(const rdhei_plan *plan, int op, int stage);

/* Form of the MED recovery wavefront.  cols = 64, 128 (default) or 256: tiles of 32
 * rows x cols columns, one warp each, taken in anti-diagonal order over all images;
 * narrow tiles give more tiles per anti-diagonal, wide ones fewer idle lanes in each
 * tile's diagonal ramp.  cols = 0: the row-band pipeline, one CTA of 16 warps per image,
 * each warp a 32-row band running a few dozen steps behind the band above (shorter
 * critical path per image, less parallelism across images).  Call after
 * rdhei_plan_create and BEFORE rdhei_plan_workspace_size / rdhei_plan_upload (it
 * changes the layout).  Returns RDHEI_EINVAL for another value or an uploaded plan. */
int rdhei_plan_set_wave_cols(rdhei_plan *plan, int cols);

/* Free launch parameters of a plan (the autotuner's knobs; results do not depend on them):
 *   RDHEI_PARAM_EXTRACT_ROWS  rows of a 64-row strip that one rdhei_decode extraction CTA
 *                             handles: 64, 32, 16, 8 or 4; 0 = chosen per batch (whole
 *                             strips, or 16 rows when the batch has fewer than 4 strips
 *                             per SM).
 *                             Takes effect at the next run.
 *   RDHEI_PARAM_ENC_SPLIT     CTAs that share one tile row of rdhei_label_encrypt's gather:
 *                             1..64; 0 = chosen per batch (more for small batches).  Takes
 *                             effect at the next run.
 *   RDHEI_PARAM_WAVE_COLS     as rdhei_plan_set_wave_cols (before upload only).
 * rdhei_plan_set_param returns RDHEI_EINVAL for an unknown parameter or value;
 * rdhei_plan_get_param returns the value in effect (the chosen one for 0), -1 if unknown. */
enum rdhei_param { RDHEI_PARAM_WAVE_COLS = 1, RDHEI_PARAM_EXTRACT_ROWS = 2, RDHEI_PARAM_ENC_SPLIT = 3 };
int rdhei_plan_set_param(rdhei_plan *plan, int param, int value);
int rdhei_plan_get_param(rdhei_plan *plan, int param);

/* ---------------------------------------------------------------------------------
 * Security and quality statistics (Sec. IV-C, Tab. analysis; PSNR and SSIM of the
 * reconstructed image, Sec. IV) for a batch of 8-bit images:
 *   entropy  H(a) = -sum_v P(v) log2 P(v), P = grey-level histogram of a / (H W),
 *            with 0 log2 0 = 0;
 *   chi2     256 (H W) sum_v (P(v) - 1/256)^2 -- the printed formula, i.e. Pearson's
 *            statistic against equal counts (about 255 for a uniform image; the
 *            paper's table lists values near its square root);
 * and, when b is given (same size):
 *   NPCR     100 * #{pixels with a != b} / (H W).  The printed indicator reads
 *            "equal", which the paper's own table values (about 99.6 % between an
 *            image and its encryption) rule out;
 *   UACI     100 * sum |a - b| / (255 H W);
 *   PSNR     10 log10(255^2 / MSE), MSE = sum (a - b)^2 / (H W); +inf when a == b;
 *   SSIM     only with RDHEI_STATS_SSIM: Wang et al. 2004 with an 11 x 11 Gaussian
 *            window (sigma 1.5, weights summing to 1), C1 = (0.01 * 255)^2,
 *            C2 = (0.03 * 255)^2, averaged over every window position inside the
 *            image; NaN when H or W is below 11 or the flag is not set.  The paper
 *            reports SSIM without defining it; this is the standard definition.
 * Without b, n_diff / sum_abs / sum_sq are 0 and npcr, uaci, psnr, ssim are NaN.
 * Exact integers: hist, n_diff, sum_abs, sum_sq.  entropy, chi2, npcr, uaci and psnr
 * are fp64 functions of them.  SSIM's local moments are fp32 (pixels centred at 128),
 * the window average fp64; its error against an fp64 evaluation is below 1e-4.
 *
 * Ownership: a, b and out are device memory owned by the caller; out must be 8-byte
 * aligned.  The workspace (256-byte aligned device memory of at least
 * rdhei_stats_workspace_size bytes) is scratch for the call.  The call copies its
 * descriptors to the workspace and waits for that copy, then launches two kernels
 * without waiting.  Errors: RDHEI_EINVAL (bad sizes, H * W > 2^31, null or misaligned
 * pointers), RDHEI_ESPACE (workspace too small), RDHEI_ECUDA. */
#define RDHEI_STATS_SSIM 1u

typedef struct rdhei_stats {
    uint32_t hist[256];
    uint64_t n_diff;      /* pixels where a != b */
    uint64_t sum_abs;     /* sum |a - b| */
    uint64_t sum_sq;      /* sum (a - b)^2 */
    double entropy, chi2, npcr, uaci, psnr, ssim;
} rdhei_stats;

typedef struct rdhei_stats_job {
    int32_t H, W;
    uint32_t flags;       /* RDHEI_STATS_SSIM or 0 */
    uint32_t reserved;
    const uint8_t *a;     /* device image, row-major H x W */
    const uint8_t *b;     /* device image compared with a, or NULL */
    rdhei_stats *out;     /* device */
} rdhei_stats_job;

size_t rdhei_stats_workspace_size(const rdhei_stats_job *jobs, int n);
int rdhei_image_stats(const rdhei_stats_job *jobs, int n, void *ws, size_t ws_bytes, void *stream);

/* The same call split for repeated use: create validates the jobs and uploads their
 * descriptors into the workspace (host-synchronous, like rdhei_plan_upload); run
 * issues one memset and the kernels only (capturable into a CUDA graph), writing
 * every job's out again; stage 0 is the histogram / pair-sum pass, stage 1 the SSIM
 * stencil.  The workspace and the images must stay valid while the plan is used;
 * destroy frees the host-side object only. */
typedef struct rdhei_stats_plan rdhei_stats_plan;
int rdhei_stats_plan_create(const rdhei_stats_job *jobs, int n, void *ws, size_t ws_bytes, void *stream,
                            rdhei_stats_plan **plan);
int rdhei_stats_plan_run(rdhei_stats_plan *plan, void *stream);
int rdhei_stats_plan_run_stage(rdhei_stats_plan *plan, int stage, void *stream);
void rdhei_stats_plan_destroy(rdhei_stats_plan *plan);

/* ---------------------------------------------------------------------------------
 * LMR side information (Sec. III-B-1, "Maps generation, rotation, and compression"
 * and "Maps embedding"; Sec. III-B-2/3, the hider and receiver read it back).  The
 * paper compresses rot(eta) and rot(l) with JBIG-KIT and writes the concatenation
 * into the first MSB plane; when it does not fit into H * W bits the owner moves to
 * the next most optimal b.  These HOST functions are a JBIG-style replacement of this
 * project's design:
 *   context   10 causal neighbours: row y-2 at x-1, x, x+1; row y-1 at x-2 .. x+2;
 *             row y at x-2, x-1 (most significant context bit first); outside = 0;
 *   model     per context counts c0 = c1 = 1 at the start, +2 per coded symbol;
 *             when c0 + c1 > 8192 both become (c >> 1) | 1;
 *   coder     binary arithmetic coding (Witten, Neal, Cleary 1987), 32-bit low/high,
 *             symbol 0 = the lower floor(range * c0 / (c0 + c1)) values, two
 *             terminating bits, MSB-first bytes zero-padded.
 * Container (the first side_nbits bits of the first MSB plane, i.e. bit 7 of pixels
 * 0 .. side_nbits - 1 of the rotated image): byte 0 = b; bytes 1..4, 5..8 = byte
 * lengths of the rot(eta) and rot(l) streams, big-endian; then both streams.
 *
 * All buffers here are HOST memory; bitmaps are H * W bits in the stream convention.
 * rdhei_lmr_side_pack: per job, compress eta_bits and map_bits (for the job's b) into
 *   side (capacity floor(H * W / 8) bytes); status RDHEI_ECAPACITY when the container
 *   does not fit (the caller tries its next b), RDHEI_EINVAL for bad arguments.
 * rdhei_lmr_side_unpack: per job, read b and both maps from a first-MSB plane
 *   (plane: ceil(H * W / 8) bytes); status RDHEI_EINVAL for a malformed container.
 * Both spread the jobs over `threads` host threads (0 = all cores) and return
 * RDHEI_EINVAL only for a bad job array; per-job results are in status.
 * rdhei_msb_plane (DEVICE, asynchronous on stream): bit 7 of every pixel of a device
 *   image, packed into out_bits (4-byte aligned, ceil(H * W / 32) words). */
typedef struct rdhei_side_pack_job {
    int32_t H, W;
    int32_t b;                /* in: the b whose location map is map_bits (2..8) */
    int32_t status;           /* out */
    const uint8_t *eta_bits;  /* in: rot(eta), H * W bits */
    const uint8_t *map_bits;  /* in: rot(l_b), H * W bits */
    uint8_t *side;            /* out: container, floor(H * W / 8) bytes available */
    uint64_t side_nbits;      /* out: container length in bits (0 on failure) */
} rdhei_side_pack_job;

typedef struct rdhei_side_unpack_job {
    int32_t H, W;
    int32_t b;                /* out */
    int32_t status;           /* out */
    const uint8_t *plane;     /* in: first MSB plane, ceil(H * W / 8) bytes */
    uint8_t *eta_bits;        /* out: rot(eta), ceil(H * W / 8) bytes */
    uint8_t *map_bits;        /* out: rot(l_b), ceil(H * W / 8) bytes */
} rdhei_side_unpack_job;

/* Eq. optimal_b as an ordered list, for an owner's fit loop that moves to the "next
 * most optimal" b when its compressed maps do not fit (Sec. III-B-1): the candidate b
 * (EMR 2..7, LMR 2..8) by decreasing capacity -- b * zeros(b) for EMR, (b - 1) *
 * zeros(b) for LMR, zeros(b) = sum over t >= b of hist[t] (rdhei_info.hist) -- ties to
 * the smaller b; order[0] is the b that rdhei_label_encrypt chooses with job.b = 0.
 * HOST function.  Returns the number of candidates (6 or 7), or -1 for a null pointer
 * or a bad variant. */
int rdhei_b_candidates(const uint32_t hist[9], int variant, int32_t order[7], uint64_t capacity[7]);

int rdhei_bilevel_encode(const uint8_t *bits, int H, int W, uint8_t *out, size_t cap, size_t *len);
int rdhei_bilevel_decode(const uint8_t *in, size_t len, int H, int W, uint8_t *bits);
int rdhei_lmr_side_pack(rdhei_side_pack_job *jobs, int n, int threads);
int rdhei_lmr_side_unpack(rdhei_side_unpack_job *jobs, int n, int threads);
int rdhei_msb_plane(const uint8_t *src, int H, int W, uint8_t *out_bits, void *stream);
size_t rdhei_side_pack_job_size(void);
size_t rdhei_side_unpack_job_size(void);

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
 *   Stream capture: a call on a stream that is being captured returns RDHEI_EINVAL
 *     and enqueues nothing (each call uploads its descriptor from a host stack buffer).
 *   Sharing: every call uses the same array and it keeps the last call's contents;
 *     what must start at zero is cleared on each call.  Calls whose work overlaps on
 *     the GPU (other streams, other threads) race: order them on one stream.
 *   Device-side errors (the checked build's index checks) reach info->status, which
 *     the call's last kernel sets (0 when none).
 *   Returns RDHEI_EINVAL for bad arguments, RDHEI_ECUDA for a failed CUDA call. */
#define RDHEI_NOALLOC_MAX_PIXELS (1u << 24)
int rdhei_extract_noalloc(const rdhei_job *job, void *stream);

/* Measurement probes (the paper has no counterpart: they measure this GPU's ceilings
 * for the roofline of the path's kernels, which are bound by integer work).
 * rdhei_probe_alu: `blocks` CTAs of 256 threads, each thread running `iters` iterations
 *   of 8 independent chains of one XOR (LOP3) and one rotation (SHF): 16 integer/logic-
 *   pipe operations per thread and iteration.  out: device, blocks * 256 words.
 * rdhei_probe_keystream: `blocks` CTAs of 256 threads, each thread computing
 *   `per_thread` ChaCha20 blocks of (key_job->k1, key_job->nonce1) with the block
 *   function of the path's kernels and XOR-folding them into one word: 64 keystream
 *   bytes per block.  out: device, blocks * 256 words; ws: device, 16-byte aligned, at
 *   least rdhei_probe_workspace_size() bytes (the call waits for its small upload).
 * Both are asynchronous on `stream` (time them with events); RDHEI_EINVAL for bad
 * arguments, RDHEI_ECUDA for a failed launch. */
int rdhei_probe_alu(uint32_t *out, int blocks, int iters, void *stream);
int rdhei_probe_keystream(uint32_t *out, int blocks, int per_thread, const rdhei_job *key_job, void *ws,
                          void *stream);
size_t rdhei_probe_workspace_size(void);

/* Failure-detection self-test of the bounded device-side wait that the MED
 * wavefront's tiles use on their neighbours' done flags: one warp waits until the
 * device word *flag is non-zero or limit_ns nanoseconds of %globaltimer have passed
 * (clamped to the library's 2 s bound), then writes RDHEI_OK or RDHEI_ETIMEOUT to the
 * device word *status and returns; the context stays usable either way.  flag and
 * status: device pointers, 4-byte aligned.  Asynchronous on `stream`.  Returns
 * RDHEI_EINVAL for null or misaligned pointers, RDHEI_ECUDA for a failed launch. */
int rdhei_wait_selftest(const uint32_t *flag, uint64_t limit_ns, int32_t *status, void *stream);

/* Workspace-wide device error word of the most recent call on this workspace
 * (synchronises the stream).  0 = no error, else an rdhei_status code. */
int rdhei_workspace_status(void *ws, void *stream, int32_t *code);

/* The same word without synchronising: queues a 4-byte copy of the uploaded plan's
 * workspace error word to dst (pinned host or device memory, 4-byte aligned) on
 * `stream`, behind the plan's work queued there; dst holds the code once the stream
 * reaches the copy.  Returns RDHEI_EINVAL for a null or misaligned dst or a plan not
 * uploaded, RDHEI_ECUDA for a failed copy. */
int rdhei_plan_copy_status(const rdhei_plan *plan, int32_t *dst, void *stream);

/* sizeof(rdhei_job) and sizeof(rdhei_info), for bindings that build them by hand. */
size_t rdhei_job_size(void);
size_t rdhei_info_size(void);
size_t rdhei_stats_size(void);
size_t rdhei_stats_job_size(void);

/* Library version and build target, e.g. "rdhei 0.1 sm_103a". */
const char *rdhei_version(void);

/* Build options of this library: RDHEI_BUILD_CHECKED is set in the checked build
 * (compiled with -DRDHEI_CHECK), whose kernels test their data-dependent indexes
 * (tile-map targets, slot-buffer and output-word positions) before each access; a
 * failing test skips the access and the call returns RDHEI_EBOUNDS.  The normal build
 * returns 0 and carries no checks. */
#define RDHEI_BUILD_CHECKED 1
int rdhei_build_flags(void);

#ifdef __cplusplus
}
#endif
#endif /* RDHEI_H */
