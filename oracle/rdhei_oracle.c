/*
 * rdhei_oracle.c -- CPU oracle for the multi-MSB replacement RDHEI method
 * (EMR-RDHEI and the per-pixel stages of LMR-RDHEI, arXiv 2302.07992).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously literal
 * restatement of the paper that the CUDA path is checked against.  Only the
 * tests, the smoke check and the CPU-baseline leg of the benchmark may load it;
 * the product library never links or calls it, and it shares no code, header,
 * table or constant with the CUDA sources.
 *
 * Every routine follows the paper's own step order and notation:
 *   - keystream s / z2 .......... Sec. III-A-1 "Secret key generation"; the paper
 *                                 asks for any cryptographically secure stream
 *                                 cipher; ChaCha20 (RFC 8439) is the one used here.
 *   - location maps ............. Sec. III-A-1a, Eqs. (gliding1), (gliding2)
 *   - choice of b ............... Eq. (optimal_b); LMR range b in [2,8] (Sec. III-B)
 *   - first MSB map eta ......... Eq. (MSB_map)
 *   - block rotation ............ Eq. (roration), Fig. (blocks)
 *   - encryption ................ Eq. (image_encryption)
 *   - EMR map embedding ......... Sec. III-A-1 "Location map embedding"
 *   - data hiding ............... Sec. III-A-2 (EMR), Sec. III-B-2 (LMR)
 *   - extraction ................ Sec. III-A-3, "receiver has only K2"
 *   - de-rotation + recovery .... Sec. III-A-3, "receiver has only K1", Eq. (roration2);
 *                                 Sec. III-B-3 for LMR
 *
 * Readings where the paper is silent or garbled are listed in the design notes
 * and repeated at the routine that takes them.  Nothing here is blocked,
 * fused or reordered for speed.
 *
 * Bit-stream convention (payload, extracted bits, packed maps, side bits and
 * the K2 keystream z2): bit k of a stream is bit (7 - k%8) of byte k/8, i.e.
 * streams are read most-significant bit first.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_EMR 0
#define ORC_LMR 1
/* Variants 2 and 3 are EMR and LMR with the MED predictor of the paper's related
 * work (Sec. II) in place of the glide; bit 1 of the variant selects the predictor,
 * bit 0 the EMR / LMR layout. */
#define ORC_MED 2
#define ORC_BASE(v) ((v) & 1)

/* ------------------------------------------------------------------------ */
/* ChaCha20 block function, written from RFC 8439 Sec. 2.1-2.3.             */
/* ------------------------------------------------------------------------ */

static uint32_t orc_rotl(uint32_t v, int c) { return (v << c) | (v >> (32 - c)); }

static uint32_t orc_le32(const uint8_t *p)
{
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

static void orc_quarter(uint32_t *x, int a, int b, int c, int d)
{
    x[a] += x[b]; x[d] ^= x[a]; x[d] = orc_rotl(x[d], 16);
    x[c] += x[d]; x[b] ^= x[c]; x[b] = orc_rotl(x[b], 12);
    x[a] += x[b]; x[d] ^= x[a]; x[d] = orc_rotl(x[d], 8);
    x[c] += x[d]; x[b] ^= x[c]; x[b] = orc_rotl(x[b], 7);
}

/* One 64-byte ChaCha20 block for (key, counter, nonce). */
void orc_chacha20_block(const uint8_t key[32], uint32_t counter, const uint8_t nonce[12], uint8_t out[64])
{
    uint32_t state[16], work[16];
    int i;
    state[0] = 0x61707865u; /* "expa" */
    state[1] = 0x3320646eu; /* "nd 3" */
    state[2] = 0x79622d32u; /* "2-by" */
    state[3] = 0x6b206574u; /* "te k" */
    for (i = 0; i < 8; i++) state[4 + i] = orc_le32(key + 4 * i);
    state[12] = counter;
    for (i = 0; i < 3; i++) state[13 + i] = orc_le32(nonce + 4 * i);
    for (i = 0; i < 16; i++) work[i] = state[i];
    for (i = 0; i < 10; i++) {           /* 20 rounds = 10 column+diagonal pairs */
        orc_quarter(work, 0, 4, 8, 12);
        orc_quarter(work, 1, 5, 9, 13);
        orc_quarter(work, 2, 6, 10, 14);
        orc_quarter(work, 3, 7, 11, 15);
        orc_quarter(work, 0, 5, 10, 15);
        orc_quarter(work, 1, 6, 11, 12);
        orc_quarter(work, 2, 7, 8, 13);
        orc_quarter(work, 3, 4, 9, 14);
    }
    for (i = 0; i < 16; i++) {
        uint32_t v = work[i] + state[i];
        out[4 * i + 0] = (uint8_t)(v);
        out[4 * i + 1] = (uint8_t)(v >> 8);
        out[4 * i + 2] = (uint8_t)(v >> 16);
        out[4 * i + 3] = (uint8_t)(v >> 24);
    }
}

/* Bytes [0, nbytes) of the ChaCha20 key stream, block counter starting at 0.
 * The image keystream s(i, j) is this stream reshaped to H x W in raster order
 * ("reshaped into the input image's size", Sec. "Secret key generation"). */
void orc_keystream(const uint8_t key[32], const uint8_t nonce[12], uint64_t nbytes, uint8_t *out)
{
    uint8_t blk[64];
    uint64_t pos = 0;
    uint32_t counter = 0;
    while (pos < nbytes) {
        uint64_t take = nbytes - pos < 64 ? nbytes - pos : 64;
        orc_chacha20_block(key, counter, nonce, blk);
        memcpy(out + pos, blk, (size_t)take);
        pos += take;
        counter++;
    }
}

/* ------------------------------------------------------------------------ */
/* Bit-stream helpers (MSB-first within each byte).                          */
/* ------------------------------------------------------------------------ */

static int orc_get_bit(const uint8_t *stream, uint64_t k)
{
    return (stream[k >> 3] >> (7 - (int)(k & 7))) & 1;
}

static void orc_put_bit(uint8_t *stream, uint64_t k, int v)
{
    uint8_t m = (uint8_t)(1u << (7 - (int)(k & 7)));
    if (v) stream[k >> 3] |= m; else stream[k >> 3] &= (uint8_t)~m;
}

/* ------------------------------------------------------------------------ */
/* Location map generation, Eqs. (gliding1), (gliding2).                     */
/*                                                                          */
/* Omega starts at the first pixel of each row and that pixel is labelled 1. */
/* Gliding along the row (the N / width axis), a pixel whose top b bits equal */
/* those of Omega is redundant (label 0); otherwise it is labelled 1 and      */
/* becomes the new Omega.                                                     */
/* Readings: the text says equal MSBs give label 0 although the printed       */
/* indicator in Eq. (gliding1) reads the other way -- the text and Eq.        */
/* (gliding2) agree, so equal -> 0.  "[1, k+1] MSBs" with b = k + 2 is read as */
/* the top b bits, which exact recovery of b replaced bits requires.          */
/* ------------------------------------------------------------------------ */
void orc_glide_labels(const uint8_t *I, int H, int W, int b, uint8_t *L)
{
    int i, j;
    for (i = 0; i < H; i++) {
        int omega = I[(size_t)i * W] >> (8 - b);
        L[(size_t)i * W] = 1;
        for (j = 1; j < W; j++) {
            int phi = I[(size_t)i * W + j] >> (8 - b);
            if (phi == omega) {
                L[(size_t)i * W + j] = 0;
            } else {
                L[(size_t)i * W + j] = 1;
                omega = phi;
            }
        }
    }
}

/* Label histogram.  For every b in 1..8 the b-MSB location map is generated by
 * the glide above; a pixel's multi-MSB label t is the number of those maps in
 * which it is redundant (the maps are nested, so t is the largest such b).
 * hist[t] counts pixels with label t, t = 0..8.  zeros(b) = sum_{t >= b} hist[t]. */
void orc_label_hist(const uint8_t *I, int H, int W, uint32_t hist[9])
{
    size_t n = (size_t)H * W, p;
    uint8_t *L = (uint8_t *)malloc(n ? n : 1);
    uint8_t *t = (uint8_t *)calloc(n ? n : 1, 1);
    int b;
    for (b = 1; b <= 8; b++) {
        orc_glide_labels(I, H, W, b, L);
        for (p = 0; p < n; p++) if (L[p] == 0) t[p]++;
    }
    for (b = 0; b < 9; b++) hist[b] = 0;
    for (p = 0; p < n; p++) hist[t[p]]++;
    free(L);
    free(t);
}

/* Eq. (optimal_b): pick b maximising (capacity per redundant pixel) x #zeros(b).
 * EMR: b in [2,7], b bits per redundant pixel.  LMR: b in [2,8], b-1 bits per
 * redundant pixel (the first MSB plane is reserved, Sec. III-B-2).
 * Ties go to the smallest b (the paper does not say). */
int orc_choose_b(int variant, const uint32_t hist[9])
{
    int b, best_b = 2, hi;
    variant = ORC_BASE(variant);
    hi = variant == ORC_EMR ? 7 : 8;
    uint64_t best = 0;
    for (b = 2; b <= hi; b++) {
        uint64_t zeros = 0, cap;
        int t;
        for (t = b; t <= 8; t++) zeros += hist[t];
        cap = (uint64_t)(variant == ORC_EMR ? b : b - 1) * zeros;
        if (b == 2 || cap > best) { best = cap; best_b = b; }
    }
    return best_b;
}

/* ------------------------------------------------------------------------ */
/* Related-work predictor (not the paper's method): the median edge detector  */
/* (MED, the LOCO-I predictor) that Sec. II quotes for Puyang et al.'s two-MSB  */
/* prediction and Puteaux et al.'s recursive labelling.  With A the left, B the */
/* upper and C the upper-left neighbour:                                       */
/*   pred = min(A, B) if C >= max(A, B); max(A, B) if C <= min(A, B);          */
/*   pred = A + B - C otherwise.                                               */
/* (The first printed form compares C with min(A, B) in its second case; the   */
/* LOCO-I form quoted second, used here, compares with max in the first.)      */
/* Borders: pixel (0, 0) has no prediction; row 0 predicts from the left       */
/* neighbour, column 0 from the upper one.  EMR loses the LSB plane at the     */
/* receiver, so its prediction works on the top seven bits (v >> 1) and is     */
/* shifted back; LMR recovers exactly and predicts on all eight bits.          */
/* ------------------------------------------------------------------------ */
static int orc_med(int A, int B, int C)
{
    int mx = A > B ? A : B, mn = A < B ? A : B;
    if (C >= mx) return mn;
    if (C <= mn) return mx;
    return A + B - C;
}

/* Prediction of pixel (i, j) from image V (original at the owner, recovered at the
 * receiver); -1 for pixel (0, 0). */
static int orc_med_pred(const uint8_t *V, int W, int i, int j, int seven)
{
    int s = seven ? 1 : 0, A, B, C;
    if (i == 0 && j == 0) return -1;
    if (i == 0) return (V[j - 1] >> s) << s;
    if (j == 0) return (V[(size_t)(i - 1) * W] >> s) << s;
    A = V[(size_t)i * W + j - 1] >> s;
    B = V[(size_t)(i - 1) * W + j] >> s;
    C = V[(size_t)(i - 1) * W + j - 1] >> s;
    return orc_med(A, B, C) << s;
}

/* Multi-MSB label against the MED prediction: t = number of leading bits (of 8)
 * in which the pixel equals its prediction, 0 for pixel (0, 0).  The b-MSB map is
 * l = 1 where t < b. */
static void orc_med_t(const uint8_t *I, int H, int W, int seven, uint8_t *T)
{
    int i, j, k;
    for (i = 0; i < H; i++)
        for (j = 0; j < W; j++) {
            int pr = orc_med_pred(I, W, i, j, seven), x = I[(size_t)i * W + j], t = 0;
            if (pr >= 0)
                for (k = 7; k >= 0 && ((x >> k) & 1) == ((pr >> k) & 1); k--) t++;
            T[(size_t)i * W + j] = (uint8_t)t;
        }
}

void orc_med_labels(const uint8_t *I, int H, int W, int seven, int b, uint8_t *L)
{
    size_t n = (size_t)H * W, p;
    uint8_t *T = (uint8_t *)malloc(n ? n : 1);
    orc_med_t(I, H, W, seven, T);
    for (p = 0; p < n; p++) L[p] = T[p] < b;
    free(T);
}

void orc_med_hist(const uint8_t *I, int H, int W, int seven, uint32_t hist[9])
{
    size_t n = (size_t)H * W, p;
    uint8_t *T = (uint8_t *)malloc(n ? n : 1);
    int k;
    orc_med_t(I, H, W, seven, T);
    for (k = 0; k < 9; k++) hist[k] = 0;
    for (p = 0; p < n; p++) hist[T[p]]++;
    free(T);
}

/* ------------------------------------------------------------------------ */
/* Multi-scale block rotation, Eq. (roration) and Eq. (roration2).           */
/*                                                                          */
/* Level L uses 2^L x 2^L blocks aligned to the image origin; blocks that do  */
/* not fit entirely inside the image are left alone.  A block's angle is the  */
/* sum of the keystream bytes s over the block, mod 4, times 90 degrees.      */
/* Readings: levels run L = lmin..n with n = floor(log2(min(H, W))) (the      */
/* printed n = min(floor(M/2), floor(N/2)) cannot be meant: for 512 x 512 the */
/* paper uses block sizes 2^1..2^9); the printed summation bounds include one */
/* row/column too many and are read as half-open; s is summed on the fixed,  */
/* unrotated grid; the rotation is counter-clockwise (numpy.rot90).  Encoding */
/* applies levels in ascending order, decoding in descending order with the  */
/* inverse angle (4 - a) mod 4.                                               */
/* ------------------------------------------------------------------------ */

int orc_levels(int H, int W)
{
    int m = H < W ? H : W, n = 0;
    while ((2 << n) <= m) n++;
    return n; /* largest n with 2^n <= min(H, W) */
}

/* Angle of block (C1, C2) at level L: (sum of s over the block) mod 4. */
int orc_block_angle(const uint8_t *s, int H, int W, int L, int C1, int C2)
{
    int B = 1 << L, i, j;
    uint64_t sum = 0;
    (void)H;
    for (i = C1 * B; i < (C1 + 1) * B; i++)
        for (j = C2 * B; j < (C2 + 1) * B; j++)
            sum += s[(size_t)i * W + j];
    return (int)(sum % 4);
}

/* Rotate the B x B block with top-left corner (r0, c0) of plane P by 90
 * degrees counter-clockwise, once: new(i, j) = old(j, B-1-i). */
static void orc_rot90_once(uint8_t *P, int W, int r0, int c0, int B, uint8_t *tmp)
{
    int i, j;
    for (i = 0; i < B; i++)
        for (j = 0; j < B; j++)
            tmp[i * B + j] = P[(size_t)(r0 + i) * W + c0 + j];
    for (i = 0; i < B; i++)
        for (j = 0; j < B; j++)
            P[(size_t)(r0 + i) * W + c0 + j] = tmp[j * B + (B - 1 - i)];
}

/* Apply the multi-scale rotation to nplanes planes of size H x W in place.
 * direction 0: encode (levels lmin..n ascending, angle a);
 * direction 1: decode (levels n..lmin descending, angle (4 - a) mod 4). */
void orc_rotate(uint8_t **planes, int nplanes, int H, int W, const uint8_t *s, int lmin, int direction)
{
    int n = orc_levels(H, W);
    int step, L, C1, C2, q, k, pl;
    uint8_t *tmp;
    if (lmin < 1) lmin = 1;
    if (n < lmin) return;
    tmp = (uint8_t *)malloc((size_t)1 << (2 * n));
    for (step = 0; step <= n - lmin; step++) {
        L = direction == 0 ? lmin + step : n - step;
        for (C1 = 0; C1 < (H >> L); C1++) {
            for (C2 = 0; C2 < (W >> L); C2++) {
                int a = orc_block_angle(s, H, W, L, C1, C2);
                q = direction == 0 ? a : (4 - a) % 4;
                for (pl = 0; pl < nplanes; pl++)
                    for (k = 0; k < q; k++)
                        orc_rot90_once(planes[pl], W, C1 << L, C2 << L, 1 << L, tmp);
            }
        }
    }
    free(tmp);
}

/* Effective smallest rotation level: 0 -> variant default (EMR 1; LMR 4, the
 * 2^4 blocks the paper adopts for 512 x 512); clamped so that at least the
 * top level rotates whenever the image has one. */
int orc_effective_lmin(int variant, int lmin, int H, int W)
{
    int n = orc_levels(H, W);
    if (lmin <= 0) lmin = ORC_BASE(variant) == ORC_EMR ? 1 : 4;
    if (n >= 1 && lmin > n) lmin = n;
    return lmin;
}

/* ------------------------------------------------------------------------ */
/* Encoding phase (content owner): Sec. III-A-1 (EMR) and III-B-1 (LMR).     */
/* ------------------------------------------------------------------------ */

/* Inputs: I (H x W), keys.  b_req = 0 chooses b by Eq. (optimal_b).
 * Outputs: enc (H x W); map_bits / eta_bits (rotated l and eta, packed, may be
 * NULL); hist[9]; *b_out; *cap_out = payload capacity in bits.
 * LMR: the first side_nbits pixels (raster order) of the encrypted image get
 * bit 7 := side bit (the compressed maps); side_bits may be NULL. */
int orc_label_encrypt(int variant, int b_req, int lmin, int rot_enable,
                      const uint8_t k1[32], const uint8_t nonce1[12],
                      const uint8_t *I, int H, int W,
                      uint8_t *enc, uint8_t *map_bits, uint8_t *eta_bits,
                      const uint8_t *side_bits, uint64_t side_nbits,
                      uint32_t hist[9], int *b_out, uint64_t *cap_out)
{
    size_t n = (size_t)H * W, p;
    uint8_t *L, *eta, *rotI, *s;
    uint8_t *planes[3];
    int b, t, med = variant & ORC_MED;
    uint64_t zeros = 0;

    variant = ORC_BASE(variant);
    /* location map generation and choice of b */
    if (med) orc_med_hist(I, H, W, variant == ORC_EMR, hist);
    else orc_label_hist(I, H, W, hist);
    b = b_req > 0 ? b_req : orc_choose_b(variant, hist);
    for (t = b; t <= 8; t++) zeros += hist[t];
    *b_out = b;
    *cap_out = (uint64_t)(variant == ORC_EMR ? b : b - 1) * zeros;

    L = (uint8_t *)malloc(n ? n : 1);
    eta = (uint8_t *)malloc(n ? n : 1);
    rotI = (uint8_t *)malloc(n ? n : 1);
    s = (uint8_t *)malloc(n ? n : 1);
    if (med) orc_med_labels(I, H, W, variant == ORC_EMR, b, L);
    else orc_glide_labels(I, H, W, b, L);

    /* first MSB map, Eq. (MSB_map): eta = (I AND 128) mod 127 */
    for (p = 0; p < n; p++) eta[p] = (uint8_t)((I[p] & 128) % 127);

    /* keystream s from K1 */
    orc_keystream(k1, nonce1, n, s);

    /* rotation of I, l (and eta) by the K1 angles */
    memcpy(rotI, I, n);
    planes[0] = rotI; planes[1] = L; planes[2] = eta;
    if (rot_enable)
        orc_rotate(planes, 3, H, W, s, orc_effective_lmin(variant, lmin, H, W), 0);

    /* encryption, Eq. (image_encryption) */
    for (p = 0; p < n; p++) enc[p] = rotI[p] ^ s[p];

    if (variant == ORC_EMR) {
        /* location map embedding into the LSB plane */
        for (p = 0; p < n; p++) enc[p] = (uint8_t)((enc[p] & 0xFE) | L[p]);
    } else if (side_bits) {
        /* compressed maps into the first MSB plane */
        for (p = 0; p < n && p < side_nbits; p++)
            enc[p] = (uint8_t)((enc[p] & 0x7F) | (orc_get_bit(side_bits, p) << 7));
    }

    if (map_bits) {
        memset(map_bits, 0, (n + 7) / 8);
        for (p = 0; p < n; p++) orc_put_bit(map_bits, p, L[p]);
    }
    if (eta_bits) {
        memset(eta_bits, 0, (n + 7) / 8);
        for (p = 0; p < n; p++) orc_put_bit(eta_bits, p, eta[p]);
    }
    free(L); free(eta); free(rotI); free(s);
    return 0;
}

/* LMR side information into the first MSB plane of an encrypted image. */
void orc_lmr_set_side(uint8_t *enc, uint64_t npx, const uint8_t *side_bits, uint64_t side_nbits)
{
    uint64_t p;
    for (p = 0; p < npx && p < side_nbits; p++)
        enc[p] = (uint8_t)((enc[p] & 0x7F) | (orc_get_bit(side_bits, p) << 7));
}

/* ------------------------------------------------------------------------ */
/* Data hiding phase (hider, K2 only): Sec. III-A-2 and III-B-2.             */
/* ------------------------------------------------------------------------ */

/* Label of pixel q seen by the hider / K2 receiver: EMR reads it from the LSB
 * plane, LMR from the (decompressed) rotated location map. */
static int orc_hider_label(int variant, const uint8_t *img, const uint8_t *lmr_map, uint64_t q)
{
    return ORC_BASE(variant) == ORC_EMR ? (img[q] & 1) : orc_get_bit(lmr_map, q);
}

/* Embed payload bits m[0..nbits) encrypted with the K2 stream z2.  Redundant
 * (label 0) pixels are visited in raster order; each offers b (EMR) or b-1
 * (LMR) bit slots starting at bit 7 (EMR) or bit 6 (LMR) and going down; the
 * encrypted payload fills the slots in order (reading: the paper only says the
 * MSBs of label-0 pixels are concatenated).  Slots past the payload keep the
 * encrypted image's bits.  Returns the number of bits embedded. */
uint64_t orc_embed(int variant, int b, const uint8_t k2[32], const uint8_t nonce2[12],
                   const uint8_t *enc, int H, int W, const uint8_t *lmr_map,
                   const uint8_t *payload, uint64_t nbits, uint8_t *marked)
{
    uint64_t n = (uint64_t)H * W, q, k = 0;
    int slots = ORC_BASE(variant) == ORC_EMR ? b : b - 1;
    int top = ORC_BASE(variant) == ORC_EMR ? 7 : 6;
    uint8_t *z2 = (uint8_t *)malloc((size_t)((nbits + 7) / 8 + 1));
    orc_keystream(k2, nonce2, (nbits + 7) / 8, z2);
    memcpy(marked, enc, (size_t)n);
    for (q = 0; q < n && k < nbits; q++) {
        int u;
        if (orc_hider_label(variant, enc, lmr_map, q) != 0) continue;
        for (u = 0; u < slots && k < nbits; u++) {
            int e = orc_get_bit(payload, k) ^ orc_get_bit(z2, k);
            int pos = top - u;
            marked[q] = (uint8_t)((marked[q] & ~(1u << pos)) | ((unsigned)e << pos));
            k++;
        }
    }
    free(z2);
    return k;
}

/* ------------------------------------------------------------------------ */
/* Decoding phase, receiver with K2: concatenate the MSB slots of label-0    */
/* pixels and decrypt with z2 (no de-rotation).  Writes min(max_bits,        */
/* capacity) bits, zero-filling the rest of the output bytes; returns that    */
/* count.                                                                     */
/* ------------------------------------------------------------------------ */
uint64_t orc_extract(int variant, int b, const uint8_t k2[32], const uint8_t nonce2[12],
                     const uint8_t *marked, int H, int W, const uint8_t *lmr_map,
                     uint8_t *bits_out, uint64_t max_bits)
{
    uint64_t n = (uint64_t)H * W, q, k = 0, cap = 0;
    int slots = ORC_BASE(variant) == ORC_EMR ? b : b - 1;
    int top = ORC_BASE(variant) == ORC_EMR ? 7 : 6;
    uint8_t *z2;
    for (q = 0; q < n; q++)
        if (orc_hider_label(variant, marked, lmr_map, q) == 0) cap += (uint64_t)slots;
    if (max_bits > cap) max_bits = cap;
    z2 = (uint8_t *)malloc((size_t)((max_bits + 7) / 8 + 1));
    orc_keystream(k2, nonce2, (max_bits + 7) / 8, z2);
    memset(bits_out, 0, (size_t)((max_bits + 7) / 8));
    for (q = 0; q < n && k < max_bits; q++) {
        int u;
        if (orc_hider_label(variant, marked, lmr_map, q) != 0) continue;
        for (u = 0; u < slots && k < max_bits; u++) {
            int bit = (marked[q] >> (top - u)) & 1;
            orc_put_bit(bits_out, k, bit ^ orc_get_bit(z2, k));
            k++;
        }
    }
    free(z2);
    return k;
}

/* ------------------------------------------------------------------------ */
/* Decoding phase, receiver with K1: decrypt, de-rotate, and restore the      */
/* replaced MSBs from the last non-redundant pixel of the row (omega glide).  */
/* EMR: the map is the LSB plane of the marked image and the recovered LSB is */
/* whatever decryption gives (the expected ~1/2 MSE).  LMR: map and eta come  */
/* decompressed from the side information; bit 7 is restored from eta and    */
/* bits 6..8-b from omega, which is lossless.                                 */
/* ------------------------------------------------------------------------ */
void orc_decrypt_recover(int variant, int b, int lmin, int rot_enable,
                         const uint8_t k1[32], const uint8_t nonce1[12],
                         const uint8_t *marked, int H, int W,
                         const uint8_t *lmr_map, const uint8_t *lmr_eta, uint8_t *out)
{
    size_t n = (size_t)H * W, p;
    uint8_t *s = (uint8_t *)malloc(n ? n : 1);
    uint8_t *L = (uint8_t *)malloc(n ? n : 1);
    uint8_t *eta = (uint8_t *)malloc(n ? n : 1);
    uint8_t *planes[3];
    int i, j, shift = 8 - b, med = variant & ORC_MED;
    unsigned field;

    variant = ORC_BASE(variant);
    field = variant == ORC_EMR ? ((1u << b) - 1) << shift : ((1u << (b - 1)) - 1) << shift;

    orc_keystream(k1, nonce1, n, s);
    for (p = 0; p < n; p++) {
        out[p] = marked[p] ^ s[p];                       /* XOR decryption */
        L[p] = variant == ORC_EMR ? (marked[p] & 1) : (uint8_t)orc_get_bit(lmr_map, p);
        eta[p] = variant == ORC_EMR ? 0 : (uint8_t)orc_get_bit(lmr_eta, p);
    }
    planes[0] = out; planes[1] = L; planes[2] = eta;
    if (rot_enable)
        orc_rotate(planes, 3, H, W, s, orc_effective_lmin(variant, lmin, H, W), 1);
    if (variant == ORC_LMR)
        for (p = 0; p < n; p++) out[p] = (uint8_t)((out[p] & 0x7F) | (eta[p] << 7));

    if (med) {
        /* MED variant: raster order is a causal order for the left, upper and
         * upper-left neighbours, so each prediction sees recovered pixels only */
        for (i = 0; i < H; i++)
            for (j = 0; j < W; j++) {
                size_t q = (size_t)i * W + j;
                if (!L[q]) {
                    int pr = orc_med_pred(out, W, i, j, variant == ORC_EMR);
                    out[q] = (uint8_t)((out[q] & ~field) | ((unsigned)pr & field));
                }
            }
        free(s); free(L); free(eta);
        return;
    }
    for (i = 0; i < H; i++) {
        unsigned omega = out[(size_t)i * W] & field;     /* first column is non-redundant */
        for (j = 1; j < W; j++) {
            size_t q = (size_t)i * W + j;
            if (L[q]) omega = out[q] & field;
            else out[q] = (uint8_t)((out[q] & ~field) | omega);
        }
    }
    free(s); free(L); free(eta);
}
