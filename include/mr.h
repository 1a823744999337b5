/*
 * mr.h -- C ABI of the GB300 RNS modular-exponentiation library (libmrmod.so).
 *
 * What it computes.  Batched x^e mod N for odd moduli of up to 16384 bits, RSA
 * encryption, RSA decryption through the CRT, Miller-Rabin rounds, the
 * primality test of key generation (trial division, then Miller-Rabin), RSA key
 * generation from candidate pools, and message-level encryption.  Numbers
 * are held in a Residue Number System (RNS): residues modulo pairwise coprime
 * primes below 2^31, one base B of k primes plus a second base B' of k primes.
 * Multiplication modulo N is the RNS Montgomery
 * multiplication with R = M = prod(B), which needs two base extensions per
 * product; exponentiation chains these products inside the Montgomery domain
 * ("Secrets from the GPU", Sec. 3.1; the constants that depend only on the
 * bases are computed once and kept resident on the GPU, same section).
 *
 * Conventions for every call.
 *  - Big integers are little-endian arrays of uint32_t limbs (limb 0 = least
 *    significant 32 bits).  A batch is a dense row-major array: row i starts at
 *    base + i*stride limbs; unused high limbs of a row must be zero.
 *  - Pointers documented as "device" point to memory of the context's GPU
 *    (cudaMalloc / torch tensors); "host" pointers point to ordinary memory.
 *    The caller owns every buffer it passes; the library owns only the context,
 *    the key handles and the tables behind them.
 *  - Batched calls are asynchronous on `stream` (a cudaStream_t; NULL = the
 *    legacy default stream).  They return after the work is enqueued; results
 *    and per-item status bytes are valid once the stream reaches that point.
 *    Scratch memory is taken from a stream-ordered pool owned by the context.
 *  - The call-level return value reports argument, setup and launch errors;
 *    mr_last_error() gives a message.  Per-item problems (an input not below
 *    its modulus, for instance) are written to dev_status[i] (device, one byte
 *    per item; 0 = ok, otherwise an mr_status code) when dev_status is not NULL.
 *  - A context is not thread-safe: serialise calls on one context.
 *  - No C++ exception crosses this interface.
 *
 * Size classes.  Classes up to 4096 bits run one number per group of GPU
 * lanes and support every call.  The large classes (8192 and 16384 bits) run
 * one group of 32 numbers across several thread blocks that exchange the base
 * extension's coefficients through device memory, in one cooperative launch;
 * they serve mr_modexp_batch, mr_rsa_encrypt and the halves of mr_rsa_decrypt_crt
 * (16384-bit keys: 8192-bit halves, recombined in binary by one warp per
 * decryption) and the large requests of mr_rsa_mixed.  Miller-Rabin, the prime
 * test and plans take at most 4096-bit numbers, key generation primes of at
 * most 2048 bits; larger inputs return MR_ERR_SIZE.
 */
#ifndef MR_H
#define MR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mr_ctx mr_ctx; /* opaque, library-owned */
typedef struct mr_key mr_key; /* opaque, library-owned */

typedef enum {
  MR_OK = 0,
  MR_ERR_ARG = 1,           /* bad argument (NULL pointer, zero stride, ...) */
  MR_ERR_EVEN_MODULUS = 2,  /* modulus even or below 3 */
  MR_ERR_NOT_COPRIME = 3,   /* modulus shares a factor with an RNS channel prime */
  MR_ERR_SIZE = 4,          /* modulus or operand longer than the largest size class */
  MR_ERR_RANGE = 5,         /* per item: input not below its modulus */
  MR_ERR_OOM = 6,           /* device or host allocation failed */
  MR_ERR_CUDA = 7,          /* a CUDA runtime call failed */
  MR_ERR_TIMEOUT = 8,       /* a bounded device wait ran out */
  MR_ERR_BUSY = 9,          /* admission refused (footprint limit) */
  MR_ERR_KEY = 10           /* key lacks the parts the call needs (e.g. no private CRT parts) */
} mr_status;

/* ---------------------------------------------------------------- context -- */

/* Create a context on CUDA device `device` (the device becomes current on the
 * calling thread).  *out receives the handle.  Errors: MR_ERR_ARG, MR_ERR_CUDA. */
mr_status mr_init(int device, mr_ctx **out);

/* Release the context, its keys and its device tables.  NULL is ignored. */
void mr_shutdown(mr_ctx *ctx);

/* Message of the last failing call on this context ("" when none).  The string
 * is owned by the context and valid until the next call on it. */
const char *mr_last_error(const mr_ctx *ctx);

/* Size class that holds a modulus of `bits` bits: *class_bits = L (one of 512,
 * 1024, 1536, 2048, 3072, 4096, 8192, 16384), *k = number of primes in each of
 * B and B'.
 * The primes lie below isqrt((2^64-1)/k) so that k-term dot products of
 * residues fit 64-bit accumulators, and the bases satisfy M >= 4 (k+1)^2 2^L
 * and M' >= 2 (k+1) 2^L, under which every Montgomery product stays below
 * (k+1) N and the B'->B extension is exact.  (Sec. 3.1 sizes a base as "k
 * channels hold keys of about 31k bits" and leaves the choice of primes open;
 * these bounds are our reading.)  Errors: MR_ERR_SIZE. */
mr_status mr_class_for_bits(uint32_t bits, uint32_t *class_bits, uint32_t *k);

/* -------------------------------------------------------------- key setup -- */

/* Per-modulus setup (Sec. 3.1: constants precomputed once and installed in GPU
 * memory).  N: host, n_limbs limbs.  Builds (or reuses) the class tables for
 * N's size class and the per-modulus constants (-N^-1 (M/m_i)^-1 mod m_i,
 * N M^-1 mod m'_j, the RNS forms of M mod N, M^2 mod N and 2^L M^2 mod N), copies
 * them to the device and returns a handle in *out.
 * Errors: MR_ERR_ARG, MR_ERR_EVEN_MODULUS, MR_ERR_NOT_COPRIME, MR_ERR_SIZE,
 * MR_ERR_OOM, MR_ERR_CUDA. */
mr_status mr_rns_setup(mr_ctx *ctx, const uint32_t *N, uint32_t n_limbs, mr_key **out);

/* RSA key (Sec. 3.3): the public modulus N = pq with public exponent e, and,
 * when p, q, dp, dq, qinv are all non-NULL, the private CRT parts (dp = d mod
 * (p-1), dq = d mod (q-1), qinv = q^-1 mod p).  All host arrays: N and e have
 * n_limbs / e_limbs limbs; p, q, dp, dq, qinv have half_limbs limbs each.
 * Private parts stay in device memory.  p and q must lie in one size class.
 * Errors: as mr_rns_setup, plus MR_ERR_ARG when N != p*q. */
mr_status mr_rsa_key_setup(mr_ctx *ctx, const uint32_t *N, uint32_t n_limbs, const uint32_t *e,
                           uint32_t e_limbs, const uint32_t *p, const uint32_t *q, const uint32_t *dp,
                           const uint32_t *dq, const uint32_t *qinv, uint32_t half_limbs, mr_key **out);

/* Size class (k) of the public modulus, k of the private halves (0 without
 * them), and device bytes held by the key.  Any output pointer may be NULL. */
mr_status mr_key_info(const mr_key *key, uint32_t *k, uint32_t *k_half, uint64_t *device_bytes);

/* Release a key (waits for the device to finish using it). NULL is ignored. */
mr_status mr_key_free(mr_ctx *ctx, mr_key *key);

/* ---------------------------------------------------------- batched calls -- */

/* out[i] = x[i]^e[i] mod N_i for i < n (Sec. 3.1: square-and-multiply chaining
 * RNS Montgomery multiplications, precomputation outside the loop).
 *   keys    host array of n handles (N_i = modulus of keys[i]; any mix of sizes)
 *   x       device, n rows of x_stride limbs, each x[i] < N_i (else status RANGE)
 *   e       device, n rows of e_stride limbs, any value (e = 0 gives 1 mod N_i)
 *   out     device, n rows of out_stride limbs; out_stride must hold N_i's limbs;
 *           the result is written in [0, N_i) and zero-padded
 *   dev_status  device, n bytes, or NULL (large classes write MR_ERR_TIMEOUT
 *               for items left unfinished when a bounded inter-block wait ran out)
 * Errors: MR_ERR_ARG, MR_ERR_SIZE, MR_ERR_OOM, MR_ERR_CUDA. */
mr_status mr_modexp_batch(mr_ctx *ctx, const mr_key *const *keys, size_t n, const uint32_t *x,
                          uint32_t x_stride, const uint32_t *e, uint32_t e_stride, uint32_t *out,
                          uint32_t out_stride, uint8_t *dev_status, void *stream);

/* RSA encryption c[i] = m[i]^e_i mod N_i with each key's public exponent
 * (Sec. 3.3: one exponentiation per message block).  Layout as mr_modexp_batch. */
mr_status mr_rsa_encrypt(mr_ctx *ctx, const mr_key *const *keys, size_t n, const uint32_t *m,
                         uint32_t m_stride, uint32_t *c, uint32_t c_stride, uint8_t *dev_status,
                         void *stream);

/* RSA decryption through the CRT: m_p = c^dp mod p, m_q = c^dq mod q (two
 * independent half-size exponentiations), h = qinv (m_p - m_q) mod p,
 * m = m_q + h q.  Equals c^d mod N (Sec. 3.3 defines d).  Keys need their
 * private parts (else MR_ERR_KEY); keys of up to 16384 bits.  c[i] < N_i
 * (else status RANGE and a zero output).  Layout as mr_modexp_batch. */
mr_status mr_rsa_decrypt_crt(mr_ctx *ctx, const mr_key *const *keys, size_t n, const uint32_t *c,
                             uint32_t c_stride, uint32_t *m, uint32_t m_stride, uint8_t *dev_status,
                             void *stream);

/* Message-level RSA (Sec. 3.3: a message is split into blocks of the key's
 * length, all blocks encrypted or decrypted in one pass).  A byte string of
 * len bytes is read as n_blocks = ceil(len / B) blocks of
 * B = (bits(N) - 1) / 8 bytes (the last one shorter), each block a
 * little-endian integer below N.  mr_rsa_message_blocks gives n_blocks, B and
 * the limbs per ciphertext row W = ceil(bits(N) / 32); needs no device.
 * Errors: MR_ERR_ARG (NULL key), MR_ERR_SIZE (N below 2^9). */
mr_status mr_rsa_message_blocks(const mr_key *key, size_t len, size_t *n_blocks, uint32_t *block_bytes,
                                uint32_t *row_limbs);

/* c (device, n_blocks rows of W limbs) = the blocks of msg (device, len
 * bytes) each raised to e mod N.  dev_status: n_blocks bytes or NULL.
 * Errors as mr_rsa_encrypt. */
mr_status mr_rsa_encrypt_message(mr_ctx *ctx, const mr_key *key, const uint8_t *msg, size_t len, uint32_t *c,
                                 uint8_t *dev_status, void *stream);

/* msg (device, len bytes) = the CRT decryptions of c (device, n_blocks rows
 * of W limbs, n_blocks as mr_rsa_message_blocks gives for len), written back
 * as bytes.  The key needs its private parts.  Errors as mr_rsa_decrypt_crt,
 * and MR_ERR_ARG when n_blocks does not match len. */
mr_status mr_rsa_decrypt_message(mr_ctx *ctx, const mr_key *key, const uint32_t *c, size_t n_blocks, uint8_t *msg,
                                 size_t len, uint8_t *dev_status, void *stream);

/* ------------------------------------------------------- mixed batches -- */

/* Operations of a mixed batch. */
enum { MR_OP_ENCRYPT = 0, MR_OP_DECRYPT = 1 };

/* Launch modes of a mixed batch (bit flags).
 *   0                    one kernel per (size class, window) group, one after another
 *                        on the call's stream ("per-size plain launches")
 *   MR_PLAN_CONCURRENT   the groups run at the same time, one stream each
 *   MR_PLAN_PERSISTENT   each group runs as a persistent kernel whose warps take
 *                        work from a device queue (items ordered by exponent length,
 *                        longest first), with a grid of one full GPU of resident
 *                        blocks, so that concurrent groups fill the SMs an earlier
 *                        group's tail frees
 *   MR_PLAN_GRAPH        (plans only) the launch sequence is captured once in a CUDA
 *                        graph and replayed by mr_plan_launch
 *   MR_PLAN_AUTOTUNE     before grouping, every size class of the batch that has not
 *                        been tuned on this context is tuned by mr_autotune with the
 *                        batch's item count and longest exponent of that class */
#define MR_PLAN_CONCURRENT 1u
#define MR_PLAN_PERSISTENT 2u
#define MR_PLAN_GRAPH 4u
#define MR_PLAN_AUTOTUNE 8u

/* One call over RSA requests of any sizes and keys (Sec. 3.3: encryption and
 * decryption by modular exponentiation; decryption here through the CRT):
 * out[i] = in[i]^e mod N_i when ops[i] == MR_OP_ENCRYPT, in[i]^d mod N_i when
 * ops[i] == MR_OP_DECRYPT (keys need private parts).  keys, ops: host arrays of
 * n; in, out: device rows (strides in limbs; out_stride must hold every
 * modulus); dev_status as mr_modexp_batch; flags: MR_PLAN_CONCURRENT,
 * MR_PLAN_PERSISTENT, MR_PLAN_AUTOTUNE (MR_PLAN_GRAPH is ignored).  Results do not
 * depend on the flags.  Requests whose exponentiations fall in a large class
 * (encryptions with keys above 4096 bits, decryptions whose CRT halves are above
 * 4096 bits) run first, as the class batches of mr_rsa_encrypt and
 * mr_rsa_decrypt_crt; the flags shape the launches of the others.  Errors as
 * mr_rsa_decrypt_crt. */
mr_status mr_rsa_mixed(mr_ctx *ctx, const mr_key *const *keys, const uint8_t *ops, size_t n, const uint32_t *in,
                       uint32_t in_stride, uint32_t *out, uint32_t out_stride, uint8_t *dev_status, uint32_t flags,
                       void *stream);

/* A prepared mixed batch: the same requests (same buffers, same keys) launched
 * many times, e.g. by a serving loop that refills `in` between launches.  The
 * plan owns its device work lists and scratch (allocated here, released by
 * mr_plan_free); with MR_PLAN_GRAPH its launches are one CUDA-graph launch.
 * Plans take requests of the lane-group classes only (keys of at most 4096 bits
 * for encryptions, CRT halves of at most 4096 bits for decryptions; others:
 * MR_ERR_SIZE). */
typedef struct mr_plan mr_plan;

mr_status mr_plan_create(mr_ctx *ctx, const mr_key *const *keys, const uint8_t *ops, size_t n, const uint32_t *in,
                         uint32_t in_stride, uint32_t *out, uint32_t out_stride, uint8_t *dev_status, uint32_t flags,
                         mr_plan **out_plan);

/* Enqueue one execution of the plan on `stream`. */
mr_status mr_plan_launch(mr_plan *plan, void *stream);

/* Kernels per launch, number of (class, window) groups, device bytes held, and
 * the estimated 32x32->64-bit products per launch (any pointer may be NULL). */
mr_status mr_plan_info(const mr_plan *plan, uint32_t *kernels, uint32_t *groups, uint64_t *device_bytes,
                       double *products);

/* Release a plan (waits for the device). NULL is ignored. */
void mr_plan_free(mr_plan *plan);

/* Miller-Rabin rounds (Sec. 3.2: Montgomery-domain primality test with a
 * caller-chosen number of iterations) on n candidates of one length.  For an
 * odd candidate N >= 3 and witness a, round r passes when, with N - 1 = 2^s d
 * (d odd) and y = (a mod N)^d mod N, y = 1, or y^(2^i) = N - 1 for some i < s.
 *   cand       device, n rows of n_limbs limbs (n_limbs * 32 <= 16384)
 *   witness    device, n*rounds rows of n_limbs limbs; row i*rounds+r is the
 *              witness of round r for candidate i (meant to lie in [2, N-2];
 *              any value is accepted and reduced mod N)
 *   rounds     >= 1
 *   dev_is_probable_prime  device, n bytes: 1 when every round passed, else 0
 *   dev_round_mask  device, n uint32 words or NULL: bit r set when round r
 *              passed (rounds <= 32 when given)
 * Candidates 0 and 1 and even candidates other than 2 are composite (mask 0);
 * 2 is prime (all bits set).  A candidate above 2^31 that is divisible by one of
 * the size class's channel primes is reported composite with mask 0 (it has
 * that prime as a factor; the per-witness verdicts are not evaluated for it).
 * Rows of at most 4096 bits (n_limbs <= 128): per-candidate constants (RNS
 * form of the candidate, Montgomery constants) are derived on the device; no
 * candidate leaves the GPU, and the call is asynchronous on `stream`.
 * Rows of the 8192- and 16384-bit classes (128 < n_limbs <= 512): the
 * candidates and witnesses are read back to the host, which derives each
 * candidate's constants as mr_rns_setup does; candidates of at most 4096
 * significant bits go through the lane-group kernel, the others through the
 * large-class exponentiation (y = a^d, then s - 1 in-place squarings), and the
 * verdicts are written back.  This form synchronises `stream` before it
 * returns.
 * Errors: MR_ERR_ARG, MR_ERR_SIZE, MR_ERR_OOM, MR_ERR_CUDA. */
mr_status mr_miller_rabin_batch(mr_ctx *ctx, const uint32_t *cand, uint32_t n_limbs, size_t n,
                                const uint32_t *witness, uint32_t rounds, uint8_t *dev_is_probable_prime,
                                uint32_t *dev_round_mask, void *stream);

/* Primality test of n candidates as key generation runs it: trial division by
 * the first n_primes primes (Sec. 4.3: the first 10,000 primes), then
 * Miller-Rabin rounds (Sec. 3.2, as mr_miller_rabin_batch) on the candidates
 * that pass it only; the rest skip the exponentiations.  A candidate passes
 * trial division when it is at least 2 and no listed prime other than itself
 * divides it.
 *   cand, n_limbs, n, witness, rounds   as mr_miller_rabin_batch
 *   n_primes       1..10000 (2, 3, 5, ... in order; the 10,000th is 104729)
 *   dev_verdict    device, n bytes: 0 = fails trial division, 1 = passes it and
 *                  some Miller-Rabin round fails (composite), 2 = passes both
 *                  (probable prime)
 *   dev_survivors  device, one uint32 or NULL: the number of candidates that
 *                  passed trial division
 * The trial-division tables (5.2 MB) are built and uploaded on the first call
 * of a context.  Errors: MR_ERR_ARG (n_primes out of range, n * rounds >= 2^32,
 * a NULL pointer), MR_ERR_SIZE, MR_ERR_OOM, MR_ERR_CUDA. */
mr_status mr_prime_test_batch(mr_ctx *ctx, const uint32_t *cand, uint32_t n_limbs, size_t n,
                              const uint32_t *witness, uint32_t rounds, uint32_t n_primes,
                              uint8_t *dev_verdict, uint32_t *dev_survivors, void *stream);

/* RSA key generation on the device from candidate pools (Sec. 3.3: N = pq,
 * d = e^-1 mod (p-1)(q-1); Sec. 3.1: Arazi's inversion; the primes pass the
 * test of mr_prime_test_batch with the first 10,000 primes).  For key k, p is
 * the first candidate of its p pool that is a probable prime with
 * gcd(e, p-1) = 1, q the first such candidate of its q pool with q != p;
 * then N = pq, d = Arazi(e, (p-1)(q-1)), dp = Arazi(e, p-1),
 * dq = Arazi(e, q-1) (so dp = d mod (p-1), dq = d mod (q-1)) and
 * qinv = q^-1 mod p; Arazi(e, f) = (1 + f t) / e with t = -f^-1 mod e.  The
 * private parts are written to device memory only.
 *   half_limbs  limbs of each candidate (2..128: primes of up to 4096 bits)
 *   n_keys, pool
 *   cand        device, n_keys * 2 * pool rows of half_limbs limbs: rows
 *               [2k pool, 2k pool + pool) are key k's p candidates, the next
 *               pool rows its q candidates (odd candidates of the wanted size;
 *               the caller supplies the randomness)
 *   witness, rounds   Miller-Rabin witnesses, `rounds` rows per candidate
 *               (row c * rounds + r), as mr_miller_rabin_batch
 *   e           public exponent, odd, 3 <= e < 2^32
 *   out         device, n_keys rows of 9 * half_limbs limbs: N (2H), d (2H),
 *               p, q, dp, dq, qinv (H each)
 *   dev_status  device, n_keys bytes or NULL: 0, MR_ERR_RANGE (a pool holds no
 *               usable prime; the row is zero) or MR_ERR_NOT_COPRIME (an
 *               inverse does not exist: a candidate passed the test but is
 *               not prime)
 * Errors: MR_ERR_ARG, MR_ERR_SIZE, MR_ERR_OOM, MR_ERR_CUDA. */
mr_status mr_rsa_keygen_batch(mr_ctx *ctx, uint32_t half_limbs, size_t n_keys, uint32_t pool,
                              const uint32_t *cand, const uint32_t *witness, uint32_t rounds, uint32_t e,
                              uint32_t *out, uint8_t *dev_status, void *stream);

/* Allocation-free exponentiation: out[i] = x[i]^e[i] mod N for i < n, one
 * modulus per call.  The paper has no counterpart; this entry point exists for
 * callers that cannot allocate device memory when they call it -- an engine that
 * has reserved all GPU memory for its own pool, or a latency-bound loop that must
 * not enter the CUDA allocator (which may synchronise the device or grow a pool).
 * It calls no cudaMalloc, cudaFree or other allocating routine and uploads no
 * work list: the caller passes inputs and outputs, and the kernel's only scratch
 * (its window tables) lives in a static device array of 16 MiB that every GPU
 * using the library keeps until the process exits.
 *   key     modulus of at most 2048 bits (else MR_ERR_SIZE)
 *   x, e, out, dev_status   as mr_modexp_batch (device rows), n items
 * A batch whose window tables exceed the 16 MiB array is refused with
 * MR_ERR_SIZE, and the message gives the largest batch that fits (1,792 items
 * of a 1024-bit modulus with a 32-limb exponent stride); split it.  The window
 * width follows from 32 * e_stride, not from the exponents' values (they are
 * in device memory): pass short exponents with the smallest stride that holds
 * them (one limb for e = 65537), which keeps both the tables and the work small.  The first call on a device looks up the array's device address;
 * make that first call before any stream capture.  All calls share the array
 * (it keeps the previous call's contents, which no call reads before writing),
 * so calls that overlap on the GPU -- on different streams, or from different
 * host threads -- race and must be serialised by the caller.
 * Errors: MR_ERR_ARG, MR_ERR_SIZE, MR_ERR_CUDA. */
mr_status mr_modexp_batch_noalloc(mr_ctx *ctx, const mr_key *key, size_t n, const uint32_t *x, uint32_t x_stride,
                                  const uint32_t *e, uint32_t e_stride, uint32_t *out, uint32_t out_stride,
                                  uint8_t *dev_status, void *stream);

/* Lane mappings compiled for a size class, for autotuning.  Each class is
 * compiled for one or more numbers of GPU lanes per number; *count receives
 * how many, lanes_per_number[0..min(count, capacity)) their lane counts (may
 * be NULL).  For the large classes a variant is a channel-slice width and its
 * lane count is the threads holding one number's channels (one lane in each
 * warp of each of the number's thread blocks); unless a variant is selected,
 * each call picks the one that needs the fewest estimated cooperative waves.
 * Errors: MR_ERR_SIZE (no such class). */
mr_status mr_class_variants(uint32_t class_bits, uint32_t *count, uint32_t *lanes_per_number, uint32_t capacity);

/* One lane mapping of a size class of at most 4096 bits: out[0] lanes per
 * number, out[1] threads per block, out[2] numbers per block, out[3] 1 when the
 * exponentiation kernel forms the two base extensions (Sec. 3.1: products with
 * the class's constant extension matrices) on the tensor cores, as exact
 * products of 8-bit slices, else 0.  out: host, 4 words.  Errors: MR_ERR_SIZE
 * (no such lane-group class), MR_ERR_ARG. */
mr_status mr_lane_variant_info(uint32_t class_bits, uint32_t variant, uint32_t *out);

/* Select the lane mapping later calls on this context use for a size class
 * (variant < count of mr_class_variants; variant 0 is the default).  Results do
 * not depend on the choice, only speed does.  Errors: MR_ERR_ARG, MR_ERR_SIZE. */
mr_status mr_set_variant(mr_ctx *ctx, uint32_t class_bits, uint32_t variant);

/* Result of mr_autotune. */
typedef struct {
  uint32_t variant;          /* chosen lane mapping (as for mr_set_variant) */
  uint32_t lanes_per_number; /* its lanes per number (as mr_class_variants reports) */
  uint32_t window;           /* chosen window-width cap */
  uint32_t configs;          /* configurations timed */
  double ms;                 /* device time of one call with the chosen configuration */
  double ms_default;         /* the same with variant 0 and the default window rule */
} mr_tune_result;

/* Measure, on this context's GPU, every compiled lane mapping of the size class
 * holding `class_bits`-bit moduli together with the window widths up to the
 * exponent-length optimum (at most 6, or 8 for the large classes), on a
 * synthetic batch of n_items exponentiations with exp_bits-bit exponents
 * modulo a seeded class_bits-bit modulus (one call per configuration after a
 * warm-up, best of two), and make the fastest the class's configuration on
 * this context (lane mapping as mr_set_variant; window width as a cap on the
 * default rule).  Results of later calls do not depend on the choice, only
 * their speed.  Synchronous; allocates about n_items * (class limbs * 8 +
 * exponent limbs * 4) bytes of device memory for the duration.  res may be
 * NULL.  Errors: MR_ERR_ARG (n_items or exp_bits zero, n_items > 2^20,
 * exp_bits > 65536), MR_ERR_SIZE, MR_ERR_OOM, MR_ERR_CUDA. */
mr_status mr_autotune(mr_ctx *ctx, uint32_t class_bits, uint32_t n_items, uint32_t exp_bits, mr_tune_result *res);

/* Tuning state of a size class on this context (class_bits: a class size as
 * mr_class_for_bits returns it): *variant = its lane mapping (as
 * mr_set_variant), *window_cap = the window-width cap (0: the default rule),
 * *tuned = 1 when mr_autotune or mr_set_tuning chose them.  Any pointer may be
 * NULL.  Errors: MR_ERR_ARG, MR_ERR_SIZE. */
mr_status mr_get_tuning(mr_ctx *ctx, uint32_t class_bits, uint32_t *variant, uint32_t *window_cap, uint32_t *tuned);

/* Install a tuning state (for instance one saved from mr_autotune on an earlier
 * context): variant < count of mr_class_variants, window_cap 0 (the default
 * rule) or up to 6 (8 for the large classes).  The class then counts as tuned
 * (MR_PLAN_AUTOTUNE leaves it alone).  Results do not depend on it, only speed
 * does.  Errors: MR_ERR_ARG, MR_ERR_SIZE. */
mr_status mr_set_tuning(mr_ctx *ctx, uint32_t class_bits, uint32_t variant, uint32_t window_cap);

/* --------------------------------------------------------- instrumentation -- */

/* Per-kernel timing.  While enabled, every batched call records a pair of CUDA
 * events around each kernel it launches, on the call's own stream.  Kernel
 * kinds: 0 = exponentiation (the RNS Montgomery loop), 1 = CRT recombination. */
typedef struct {
  uint32_t launches; /* kernels of this kind launched since the last read */
  double ms;         /* their summed device time (ms); 0 when timing was off */
} mr_kernel_time;

/* Turn event timing on (on != 0) or off.  Launch counting is always on. */
mr_status mr_profile_enable(mr_ctx *ctx, int on);

/* Wait for the recorded events, then return per-kind totals since the last
 * read in times[0..n_kinds) (n_kinds <= 2) and reset the counters. */
mr_status mr_profile_read(mr_ctx *ctx, mr_kernel_time *times, uint32_t n_kinds);

/* Measured integer-multiply throughput of this GPU, the denominator the
 * exponentiation kernels are compared against: a dependent-free stream of
 * 32x32 multiply-adds in every lane of every SM, timed with CUDA events on
 * `stream` (NULL = the default stream).  kind 0: mad.wide.u32 (64-bit product
 * added to a 64-bit accumulator, the instruction of the channel products and
 * base-extension dot products); kind 1: mad.lo.u32; kind 2: the same 64-bit
 * accumulation as a carry pair, mad.lo.cc.u32 + madc.hi.u32 (rate in products,
 * two instructions each); kind 3: mad.hi.u32.  *per_second receives
 * instructions (kind 2: products) per second summed over all lanes.  Takes a
 * few milliseconds of device time; allocates 8 bytes of device memory for the
 * duration.  Errors: MR_ERR_ARG (kind > 3, NULL pointer), MR_ERR_CUDA. */
mr_status mr_imad_peak(mr_ctx *ctx, uint32_t kind, void *stream, double *per_second);

/* Measured tensor-core throughput of this GPU (Sec. 3.1: the base extensions
 * are products with constant matrices, the one dense contraction of the path),
 * in operations (2 per multiply-add) per second over all SMs, timed with CUDA
 * events on `stream`.  kind 0: tcgen05.mma kind::f16 (fp16 operands in shared
 * memory, fp32 accumulator in tensor memory, M = 128, N = 256, K = 16, one CTA
 * per SM); kind 1: mma.sync m16n8k32 s8 -> s32 (the integer tensor path that
 * sm_103a offers: tcgen05 has no kind::i8 there); kind 2: mma.sync m16n8k16
 * f16 -> f32.  Allocates 64 bytes of device memory for the duration.  Errors:
 * MR_ERR_ARG, MR_ERR_TIMEOUT (a bounded completion wait ran out; the tensor
 * memory was released), MR_ERR_CUDA. */
mr_status mr_tensor_peak(mr_ctx *ctx, uint32_t kind, void *stream, double *ops_per_second);

/* One compiled variant of a large size class (8192, 16384 bits): channels per
 * thread block and base, thread blocks per group of 32 numbers, and whether its
 * two base extensions run on the tensor cores (1: fp16 slices with fp32
 * accumulation in tensor memory, exact; 0: the integer pipe).  Results do not
 * depend on the variant.  Any output pointer may be NULL.  Errors: MR_ERR_SIZE
 * (no such class), MR_ERR_ARG (not a large class, or no such variant). */
mr_status mr_big_variant_info(uint32_t class_bits, uint32_t variant, uint32_t *slice_channels, uint32_t *slices,
                              uint32_t *tensor);

/* The tensor-core operand table of a size class's base extensions, built on the
 * host (no device needed): for each channel slice of 32 output channels c and
 * each extension matrix (T1 = |M/m_i|_{m'_j} 2^64 mod m'_j, then T2 =
 * |M'/m'_j|_{m_i} 2^64 mod m_i; row = input channel, 4 x 7-bit slices of
 * every entry), the fp16 values of slice b of column j at row 32 b + j of a
 * 128-row K-major tile, in chunks of 64 input channels; layout
 * [slice][matrix][chunk][16 KB].  *count receives the number of 32-bit words
 * (two fp16 values each, the lower address in the low half); out may be NULL
 * to query it.  Errors: MR_ERR_SIZE (no such class, or an entry above 28
 * bits), MR_ERR_ARG (capacity too small). */
mr_status mr_debug_tc_slices(uint32_t class_bits, uint32_t *out, size_t capacity, size_t *count);

/* Test hook of the tensor-core operand layout: one CTA computes the exact fp32
 * product D = A * B^T with tcgen05 (A: 128 x kdim fp16, B: n x kdim fp16, both
 * row-major host arrays; D: 128 x n fp32 host array, row-major), staging both
 * operands in the K-major shared-memory layout of the tensor-core extension.
 * swap_strides = 1 exchanges the descriptor's two byte offsets (diagnosis
 * only; kdim must then be 16); swap_strides = 2 takes A from tensor memory
 * instead (row r in lane r, two fp16 values of K per 32-bit column, the lower
 * K index in the low half: the layout of the extension's resident matrix);
 * swap_strides = 3 computes the product as 0 does and reads D back with the
 * 16x256b tensor-memory load shape (the lane-group extensions' epilogue).
 * 16 <= n <= 256 (n <= 128 with swap_strides 1 or 2) and 16 <= kdim <= 64, both
 * multiples of 16.
 * Synchronises `stream`.  Errors: MR_ERR_ARG, MR_ERR_TIMEOUT, MR_ERR_CUDA. */
mr_status mr_debug_tc_mma(mr_ctx *ctx, const uint16_t *a, const uint16_t *b, uint32_t n, uint32_t kdim,
                          uint32_t swap_strides, float *d, void *stream);

/* Constant-time exponentiation schedule (the paper's square-and-multiply with
 * precomputation, Sec. 3.1, in a form whose memory addresses and branches do
 * not depend on exponent bits).  on != 0: later calls on this context, and
 * plans created while it is on, run the lane-group size classes (512 to 4096
 * bits) with fixed windows over every limb of each exponent row (leading zero
 * limbs included), a multiplication for every window (a zero digit multiplies
 * by the Montgomery form of 1), no sliding windows, and table entries read by
 * touching every entry and keeping the wanted one by masking.  Results are
 * identical; the cost is the extra multiplications and table reads.  The
 * window width is still chosen from the exponents' bit lengths, and the large
 * classes (8192, 16384 bits) keep their direct table lookups.  on == 0
 * restores the default.  Errors: MR_ERR_ARG. */
mr_status mr_set_constant_time(mr_ctx *ctx, int on);

/* Phase counters of the tensor-core form of the large classes (instrumentation,
 * off by default).  on != 0: later calls on this context add, per thread block
 * (its thread 0), the SM clock cycles spent in each phase of every RNS
 * Montgomery multiplication: 0 channel work up to the first exchange, 1 the
 * first barrier between the blocks of an item group, 2 the first extension's
 * copies and tensor-core products, 3 its epilogue, 4 channel work up to the
 * second exchange, 5 the second barrier, 6 the second extension's copies and
 * products, 7 its epilogue and the final channel work.  When out is not NULL
 * it receives the 8 sums and then the number of blocks counted (9 words),
 * after a device synchronisation, and the counters restart from zero.
 * on == 0 releases them (after reading into out, if given).  Allocates 72
 * bytes of device memory while on.  Errors: MR_ERR_ARG, MR_ERR_CUDA. */
mr_status mr_debug_big_phases(mr_ctx *ctx, int on, uint64_t *out);

/* Test hook of the large classes' bounded waits.  Later 8192/16384-bit calls on
 * this context give up a wait between thread blocks after spin_limit polls
 * (0 restores the default, about one second), and, when absent_slice >= 0, the
 * blocks of that channel slice leave at once without arriving at any wait, so
 * that the others time out: the call then completes, every item's status byte
 * is MR_ERR_TIMEOUT and the context stays usable.  absent_slice = -1 turns the
 * hook off.  Errors: MR_ERR_ARG. */
mr_status mr_debug_big_wait(mr_ctx *ctx, uint32_t spin_limit, int32_t absent_slice);

/* Test hook of the bounded completion wait of the lane-group classes' tensor-core
 * kernels (the base extensions of Sec. 3.1 as tcgen05 products).  With skip != 0,
 * later batch calls on this context (mr_modexp_batch, mr_rsa_encrypt,
 * mr_rsa_decrypt_crt and the calls built on them; not plans) launch those
 * kernels with no product issued, so every block's first completion wait runs
 * out after about one second: the call completes, every item of such a kernel
 * reports MR_ERR_TIMEOUT and the context stays usable.  skip = 0 turns the hook
 * off.  Errors: MR_ERR_ARG. */
mr_status mr_debug_lane_tc_wait(mr_ctx *ctx, int skip);

/* ------------------------------------------------------------ inspection -- */

/* Copy one precomputed table of a size class (or of a key when key != NULL) to
 * host memory, as plain residues (not the device's internal scaled form), in
 * the order of the same-named tables of the CPU model of the method.  Used by
 * tests to check the setup value by value; needs no device (ctx may be NULL
 * for class tables).  *count receives the number of uint32 words; out may be
 * NULL to query it.  Class tables: "B", "Bp" (the channel primes), "M_mi_inv"
 * (|(M/m_i)^-1|_{m_i}), "M_mi_Bp" (row i, column j: |M/m_i|_{m'_j}), "Minv_Bp",
 * "Mp_mj_inv", "Mp_mj_B" (row j, column i), "Mp_B", "M" (limbs of M), "bound"
 * (the channel-prime bound as two words, low first).  Key tables: "kxi",
 * "NMinv_Bp", "one", "r2", "r2h" (RNS vectors: B residues, then B').
 * Errors: MR_ERR_ARG (unknown name, or out too small), MR_ERR_SIZE. */
mr_status mr_debug_table(mr_ctx *ctx, uint32_t class_bits, const mr_key *key, const char *name,
                         uint32_t *out, size_t capacity, size_t *count);

/* Test hook of mr_miller_rabin_batch: run one round (witness 2) on n candidates
 * and write, per candidate, the constants the kernel derived on the device to
 * dev_out (device, n rows of 4 + 2W + 5k words, W = class limbs, k = class
 * channels): [special case code, s, bit length, 0], M mod N (W limbs),
 * M^2 mod N (W limbs), then per channel |-N^-1 (M/m_i)^-1|_{m_i} (k),
 * |N M^-1|_{m'_j} (k), |N M^-1 (M'/m'_j)^-1|_{m'_j} (k), N^-1 mod m_i (k),
 * N^-1 mod m'_j (k).  Synchronises the stream.  Errors as mr_miller_rabin_batch. */
mr_status mr_debug_mr_setup(mr_ctx *ctx, const uint32_t *cand, uint32_t n_limbs, size_t n, uint32_t *dev_out,
                            void *stream);

/* The large classes' choice of slice width (host only, no context): for a batch
 * of n_items exponentiations of class class_bits (8192 or 16384) on a GPU of
 * `sms` SMs holding ctas_per_sm blocks of every variant per SM, *variant is the
 * variant with the fewest estimated cooperative waves (waves x the variant's
 * relative time per group of 32 numbers) and *slots the groups it runs at once.
 * Errors: MR_ERR_ARG, MR_ERR_SIZE (not a large class, or nothing fits). */
mr_status mr_debug_big_variant(uint32_t class_bits, size_t n_items, uint32_t sms, uint32_t ctas_per_sm,
                               uint32_t *variant, uint32_t *slots);

/* The binary Garner block that CRT keys with halves in a large size class carry
 * (host only, no context): for primes p, q and qinv = q^-1 mod p (n_limbs limbs
 * each) and the class's limb count W: [P2: W+1 limbs][qr: W][q: W][pinv: 1] with
 * P2 = p * ceil(2^(32W) / p), qr = qinv * 2^(32(W+1)) mod p, pinv = -p^-1 mod 2^32.
 * *count receives the word count (3W + 2); out may be NULL to query it.
 * Errors: MR_ERR_ARG, MR_ERR_EVEN_MODULUS (p even). */
mr_status mr_debug_crt_bin_host(const uint32_t *p, const uint32_t *q, const uint32_t *qinv, uint32_t n_limbs,
                                uint32_t W, uint32_t *out, size_t capacity, size_t *count);

/* The trial-division tables of mr_prime_test_batch as built on the host (no
 * context, no device): 131 rows of 10,016 words: rows w < 128 hold
 * 2^(32w) mod p_j for the first 10,000 primes p_j (column j), row 128 the
 * primes (columns past 10,000 zero in these rows), then from row 129 on the
 * factors floor((2^64-1)/p_j) as consecutive little-endian word pairs.  *count
 * receives the word count; out may be NULL to query
 * it.  Errors: MR_ERR_ARG (out too small). */
mr_status mr_debug_trial_table(uint32_t *out, size_t capacity, size_t *count);

/* As mr_debug_table for the key tables of modulus N (host, n_limbs limbs),
 * computed on the host only (no context, no device).  Errors as mr_rns_setup. */
mr_status mr_debug_key_table_host(const uint32_t *N, uint32_t n_limbs, const char *name, uint32_t *out,
                                  size_t capacity, size_t *count);

#ifdef __cplusplus
}
#endif
#endif /* MR_H */
