/*
 * fhe.h -- C ABI of libfhe_gb300: the non-RNS CKKS hot path on one GB300 (sm_103a).
 *
 * Scheme: the original (non-RNS) CKKS of Cheon et al. as adopted by LibFHE
 * (Sec. 2 "Fully Homomorphic Encryption", Sec. 3 "Why Original CKKS", Sec. 6).
 * Ciphertext coefficients are single big integers modulo Q = 2^logQ, stored in
 * the radix-2^32 limb form of Sec. 4 ("The Radix Representation", 32-bit limbs)
 * and converted to RNS only inside ring products (Sec. 4 "Hybrid Representation
 * Strategy"; Sec. 5 pipeline: limb -> RNS -> NTT -> pointwise -> INTT -> Garner
 * -> limb).  The homomorphic operations follow the paper's operation list
 * (Sec. 6 "Homomorphic Operation API").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Limb layout ("SoA"): a polynomial with N coefficients of L limbs is
 *   uint32_t[L][N]: limb l of coefficient i at [l*N + i], least significant
 *   limb first, N contiguous.  L = ceil(logQ / 32).  Bits at or above logQ
 *   of the top limb are zero on every output (canonical residues in [0, Q)).
 * Ciphertext batch (the paper's CipherTensor with batch size cnum, Sec. 6
 *   "Pairwise and Broadcast Modes"): uint32_t[cnum][2][L][N]; polynomial 0 is
 *   b, polynomial 1 is a, and decryption is b + a*s (mod Q).
 * Device vs host: every pointer documented "device" must be a device pointer
 *   on the context's device; "host" pointers are read synchronously.  The
 *   caller owns all ciphertext, plaintext and workspace buffers; the library
 *   never frees them.  Keys, tables and the secret live in memory the context
 *   owns (allocated through the allocator given at creation).
 * Streams: `stream` is a cudaStream_t (NULL = legacy default stream).  Calls
 *   enqueue work and return; results are ready when the stream reaches them.
 *   Operations on one context may run on several streams only if their
 *   workspaces differ.
 * Workspace: operations that need scratch take a caller-allocated device
 *   buffer `ws` of at least fhe_workspace_bytes(...) bytes (256-byte aligned).
 * Errors: every int-returning call returns FHE_OK (0) or a negative FHE_E*
 *   code; fhe_last_error() returns a message for the calling thread.
 *   Arguments are validated before anything is enqueued; a call that fails
 *   validation has no effect.  Asynchronous CUDA errors surface as FHE_ECUDA
 *   on a later call or on fhe_sync().
 * Aliasing: `out` may alias `in` for fhe_rescale, fhe_moddown, fhe_negate,
 *   fhe_add and fhe_sub; it must not alias an input of any other operation.
 */
#ifndef FHE_GB300_H
#define FHE_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FHE_OK 0
#define FHE_EINVAL (-1)    /* bad argument (null pointer, size or range)          */
#define FHE_ENOMEM (-2)    /* the context's allocator failed                      */
#define FHE_ELEVEL (-3)    /* operand levels/ring sizes do not match the request   */
#define FHE_ENOKEY (-4)    /* no key for the requested operation (keygen missing)  */
#define FHE_ECUDA (-5)     /* a CUDA runtime call failed                           */
#define FHE_ETIMEOUT (-6)  /* a bounded device-side wait gave up                   */
#define FHE_EWORKSPACE (-7)/* workspace null, too small or misaligned              */

#define FHE_SCHEME_CKKS 0
#define FHE_SCHEME_BGV 1

/* Operation codes for fhe_workspace_bytes. */
#define FHE_OP_MULT 1      /* fhe_mult_relin / fhe_mult_relin_rescale  */
#define FHE_OP_ROTATE 2    /* fhe_rotate, fhe_rotate_hoisted, fhe_conjugate */
#define FHE_OP_ENCRYPT 3   /* fhe_encrypt, fhe_encrypt_inject          */
#define FHE_OP_DECRYPT 4   /* fhe_decrypt                              */
#define FHE_OP_KEYGEN 5    /* key generation scratch (informational)   */
#define FHE_OP_RING_MUL 6  /* fhe_ring_mul with logQ = max operand bits */
#define FHE_OP_MULT_RAGGED 7 /* fhe_mult_relin_rescale_ragged, logQ = the largest level */
#define FHE_OP_MULT_PLAIN 8  /* fhe_mult_plain                           */
#define FHE_OP_ENCODE 9      /* fhe_ckks_encode / fhe_ckks_decode (logQ ignored) */

typedef struct fhe_ctx fhe_ctx;

/* Device allocator used for everything the context owns (keys, tables).
 * alloc returns a device pointer aligned to 256 bytes, or NULL.  With both
 * NULL the context uses cudaMalloc / cudaFree. */
typedef void* (*fhe_alloc_fn)(size_t bytes, void* user);
typedef void (*fhe_free_fn)(void* ptr, size_t bytes, void* user);

typedef struct {
  int32_t scheme; /* FHE_SCHEME_CKKS or FHE_SCHEME_BGV                                */
  int32_t logN;   /* ring X^N + 1, N = 2^logN, 3 <= logN <= 16 (Sec. 6 parameter n)   */
  int32_t logQ;   /* CKKS: top modulus Q = 2^logQ (Sec. 6 log q).  BGV: the bit length
                     of the top modulus Q_L = q0 r^L (checked)                         */
  int32_t logP;   /* special modulus P = 2^logP of the switching keys                 */
  int32_t crt;    /* RNS -> limb reconstruction: FHE_CRT_DIRECT (0, default),
                     FHE_CRT_GARNER (1, the mixed-radix form of Sec. 2 Eq. garner_mrc)
                     FHE_CRT_DIRECT_INT (2) or FHE_CRT_DIRECT_CVT (3); all give
                     identical results                                              */
  int32_t bgv_levels; /* BGV: top level L of the chain Q_l = q0 r^l (0 for CKKS)      */
  uint32_t t;         /* BGV: plaintext modulus, odd, 3 <= t < 2^31 (0 for CKKS)      */
  uint64_t bgv_q0;    /* BGV: odd, = 1 mod t                                         */
  uint64_t bgv_r;     /* BGV: odd, = 1 mod t, 2^8 < r < 2^62                           */
  int32_t hamming_weight; /* secret of fhe_keygen: 0 = uniform ternary, h > 0 = exactly h
                             nonzero coefficients in {-1, 1} (sparse secret, HEAAN's HWT)  */
  double sigma;       /* error standard deviation of fhe_keygen / fhe_encrypt (0 = 3.2),
                         rounded Gaussian cut at |e| <= floor(6 sigma), sigma <= 10        */
} fhe_params;

#define FHE_CRT_DIRECT 0     /* exact CRT sum with a rounded quotient (Halevi-Polyakov-Shoup);
                                the dense sum runs on the fp16 tensor cores as a byte-digit
                                GEMM wherever r + 1 <= 255 and N is a multiple of 64      */
#define FHE_CRT_GARNER 1     /* Garner's mixed-radix conversion, digits in the nested order   */
#define FHE_CRT_DIRECT_INT 2 /* the direct CRT with its dense sum on the integer pipe only  */
#define FHE_CRT_DIRECT_CVT 3 /* FHE_CRT_DIRECT with the column sums always converted by
                                cvt.rni (FHE_CRT_DIRECT converts them with one exact fp32
                                addition where a host-side bound shows |sum| < 2^22)      */

typedef struct {
  uint32_t* data; /* device, uint32_t[cnum][2][L][N], L = ceil(logQ/32)               */
  int32_t cnum;   /* batch size (CipherTensor cnum, Sec. 6)                          */
  int32_t logQ;   /* CKKS: this ciphertext's modulus 2^logQ (its level), <= the top.
                     BGV: the bit length of Q_level (must match `level`)             */
  int32_t level;  /* BGV: level l of the modulus Q_l = q0 r^l (ignored for CKKS)     */
  double log_scale; /* CKKS: log2 of the scale Delta of the encrypted message.  The caller
                       sets it on encryption; every operation writes its output's scale
                       (mult: sum of the inputs', rescale by k: minus k, the rest: the
                       input's) and fhe_add / fhe_sub reject operands whose scales differ
                       by more than 1e-9 (FHE_ELEVEL).  Ignored for BGV.                   */
} fhe_ct;

/* Create a context for one ring size and modulus chain.  Computes the NTT
 * primes (30-bit, q = 1 mod 2N; Sec. 4) and the precomputed tables of
 * Sec. 5 "Precomputation" (bit-reversed psi powers and their inverses,
 * 2^(32 l) mod q_i, Garner constants [q_j^-1]_{q_k}, prod_{i<k} q_i) and
 * uploads them.  `alloc`/`free_` may both be NULL (cudaMalloc/cudaFree).
 * Uses the current CUDA device.  Returns FHE_EINVAL for out-of-range
 * parameters, FHE_ENOMEM / FHE_ECUDA on allocation or copy failure. */
int fhe_ctx_create(const fhe_params* params, fhe_alloc_fn alloc, fhe_free_fn free_, void* alloc_user,
                   fhe_ctx** out);

/* Release everything the context owns (synchronises the device first). */
int fhe_ctx_destroy(fhe_ctx* ctx);

/* Message of the last failed call on this thread ("" if none). */
const char* fhe_last_error(void);

/* Synchronise the device and report any pending asynchronous CUDA error;
 * FHE_ETIMEOUT if a kernel's bounded wait (the tensor-core reconstruction's
 * pipeline barriers) gave up since the last call, in which case the results
 * enqueued meanwhile are invalid. */
int fhe_sync(fhe_ctx* ctx);

/* Bytes of a ciphertext batch: cnum * 2 * ceil(logQ/32) * 2^logN * 4. */
size_t fhe_ct_bytes(int logN, int logQ, int cnum);

/* Workspace bytes an operation needs for `cnum` ciphertexts at level logQ
 * (for FHE_OP_RING_MUL: logQ = the larger operand's bits).  0 on bad args. */
size_t fhe_workspace_bytes(const fhe_ctx* ctx, int op, int logQ, int cnum);

/* Key generation from a seed (Sec. 6 "Cryptographic Key Management": the secret
 * key, the public key, the relinearisation key rk, rotation keys rtk_j and, for
 * CKKS, the conjugation key ck).  Every random polynomial is drawn by the
 * library's counter-based sampler (Philox4x32-10, Salmon et al. 2011) from
 * `seed`; see fhe_sample for the streams and rules.  The secret is uniform
 * ternary, or of Hamming weight params.hamming_weight; errors are rounded
 * Gaussians of params.sigma; the uniform key parts are uniform mod 2^logQ and
 * 2^(logP + logQ) (BGV: full 32-bit limbs, then reduced mod Q and P Q).
 * rot_steps (host int[n_rot], may be NULL when n_rot = 0) lists the left
 * rotations (negative = right) to make keys for.  The keys are then as
 * fhe_keygen_inject and fhe_keygen_rotation make them from the same draws.
 * Synchronous.  The same seed always gives the same keys: use a fresh,
 * secret seed for every key set. */
int fhe_keygen(fhe_ctx* ctx, uint64_t seed, const int* rot_steps, int n_rot);

/* Key generation from caller-supplied random polynomials (host pointers), so
 * that results can be reproduced outside the library.
 * BGV: the errors are multiplied by t, Q is the top chain modulus q0 r^L and
 * a_pk / a_ev are first reduced modulo Q and P Q (any limbs are accepted).
 *   s     int8_t[N]            secret, coefficients in {-1, 0, 1}
 *   a_pk  uint32_t[Lq][N]      uniform mod Q,   Lq  = ceil(logQ/32)
 *   e_pk  int32_t[N]           small error
 *   a_ev  uint32_t[Lpq][N]     uniform mod P*Q, Lpq = ceil((logP+logQ)/32)
 *   e_ev  int32_t[N]           small error
 * Computes on the GPU pk = (-a_pk s + e_pk, a_pk) mod Q and
 * evk = (-a_ev s + e_ev + P s^2, a_ev) mod P*Q, and keeps them resident
 * (evk in NTT form over the key-switching primes).  Synchronous. */
int fhe_keygen_inject(fhe_ctx* ctx, const int8_t* s, const uint32_t* a_pk, const int32_t* e_pk, const uint32_t* a_ev,
                      const int32_t* e_ev);

/* Rotation key for left rotation by `step` slots (Sec. 6 rtk; leftrotate):
 * rtk = (-a s + e + P s(X^g), a) mod P*Q with g = 5^step mod 2N.
 * a: host uint32_t[Lpq][N], e: host int32_t[N].  Requires a key set first.
 * Replaces an existing key for the same g.  CKKS only.  Synchronous. */
int fhe_keygen_rotation(fhe_ctx* ctx, int step, const uint32_t* a, const int32_t* e);

/* Conjugation key (Sec. 6 ck, for conjugate_pairwise_into): the switching key
 * of the automorphism X -> X^(2N-1), ck = (-a s + e + P s(X^-1), a) mod P*Q.
 * Arguments as for fhe_keygen_rotation.  CKKS only.  Synchronous. */
int fhe_keygen_conjugation(fhe_ctx* ctx, const uint32_t* a, const int32_t* e);

/* Public-key encryption (encrypt_pairwise_upon, Sec. 6) of cnum plaintexts
 * with the ephemeral v and errors e0, e1 of ciphertext c drawn by the
 * library's sampler from (seed, c) (ternary v, rounded Gaussian e0, e1; see
 * fhe_sample), then as fhe_encrypt_inject.  Never reuse a seed under one key:
 * two encryptions with the same (seed, c) reveal their plaintext difference.
 * Workspace: FHE_OP_ENCRYPT. */
int fhe_encrypt(fhe_ctx* ctx, const uint32_t* pt, uint64_t seed, fhe_ct* out, void* ws, size_t ws_bytes,
                void* stream);

/* Public-key encryption with caller-supplied randomness:
 *   CKKS: out = (v pk_b + m + e0, v pk_a + e1) mod 2^out->logQ
 *   BGV:  out = (v pk_b + m + t e0, v pk_a + t e1) mod Q_{out->level}, pt canonical
 *         residues (m in [0, t) in limb 0)
 * pt: device uint32_t[cnum][L][N], each coefficient m mod 2^logQ (a signed
 * plaintext in two's complement); v: device int8_t[cnum][N] in {-1,0,1};
 * e0, e1: device int32_t[cnum][N].  out->data, out->cnum, out->logQ (and
 * out->log_scale, the plaintext's scale) set by the caller (logQ <= top).
 * FHE_ENOKEY before key generation. */
int fhe_encrypt_inject(fhe_ctx* ctx, const uint32_t* pt, const int8_t* v, const int32_t* e0, const int32_t* e1,
                       fhe_ct* out, void* ws, size_t ws_bytes, void* stream);

/* The library's sampler on the host (no GPU needed): n coefficients of the
 * stream (seed, tag0, tag1) that fhe_keygen and fhe_encrypt draw from.  Word j
 * of a stream is component j mod 4 of Philox4x32-10 (Salmon et al., SC 2011)
 * with counter (j/4 mod 2^32, j/2^34, tag0, tag1) and key (seed mod 2^32,
 * seed / 2^32).  kind:
 *   FHE_SAMPLE_UNIFORM   uint32_t[L][n] uniform mod 2^param (L = ceil(param/32));
 *                        limb l of coefficient i is word l n + i, top limb masked
 *   FHE_SAMPLE_TERNARY   int8_t[n], floor(3 w / 2^32) - 1
 *   FHE_SAMPLE_HWT       int8_t[n] with exactly param nonzero coefficients in
 *                        {-1, 1}: a partial Fisher-Yates shuffle over words 0..param-1
 *                        (swap i, i + floor((n - i) w_i / 2^32)), signs from bit 0 of
 *                        words param..2 param - 1 (odd = -1)
 *   FHE_SAMPLE_GAUSSIAN  int32_t[n] rounded Gaussian of standard deviation sigma:
 *                        the smallest k with w < T_k, T_k = floor(2^32 S_k / S_B),
 *                        S_k the in-order double sums of exp(-k^2 / (2 sigma^2)) from
 *                        k = -B, B = floor(6 sigma); B if there is none
 * Tags used by the library (tag0): 1 secret, 2 / 3 public key a / e,
 * 4 / 5 relinearisation key a / e, 6 / 7 switching key a / e with tag1 = its
 * Galois element, 8 / 9 / 10 encryption v / e0 / e1 with tag1 = the
 * ciphertext's index in the batch.  out: host memory.  FHE_EINVAL on a bad
 * kind, parameter or n (1 <= n <= 2^24). */
#define FHE_SAMPLE_UNIFORM 0
#define FHE_SAMPLE_TERNARY 1
#define FHE_SAMPLE_HWT 2
#define FHE_SAMPLE_GAUSSIAN 3
int fhe_sample(uint64_t seed, uint32_t tag0, uint32_t tag1, int kind, int n, int param, double sigma, void* out);

/* Decryption (decrypt_pairwise_upon, Sec. 6): m = [b + a s]_Q with the centred
 * reduction of Sec. 5 ("if x > Q/2, x <- x - Q").  CKKS: written as L-limb two's
 * complement (sign-extended to 32 L bits), pt_out device uint32_t[cnum][L][N].
 * BGV: m mod t of the centred value, pt_out device uint32_t[cnum][N]. */
int fhe_decrypt(fhe_ctx* ctx, const fhe_ct* in, uint32_t* pt_out, void* ws, size_t ws_bytes, void* stream);

/* Homomorphic multiplication with relinearisation (mult_pairwise_into, Sec. 6).
 * BGV: same shape modulo the odd Q_l of the operands' level, with the key-switch
 * division (y + delta)/P, delta = t [(-y) t^-1]_P (centred), so delta = 0 mod t.
 * CKKS:
 *   (d0, d1, d2) = (b1 b2, a1 b2 + a2 b1, a1 a2) mod Q    (4 forward, 3 inverse NTTs, Sec. 5)
 *   out = (d0, d1) + round(P^-1 (d2~ evk_b, d2~ evk_a) mod P Q)  (mod Q),
 * d2~ the centred representative of d2 (logQ-bit two's complement).
 * a, b: same logQ; b->cnum = a->cnum (pairwise mode) or 1 (broadcast mode: the
 * one ciphertext b multiplies every ciphertext of a, Sec. 6 "Pairwise and
 * Broadcast Modes"); out: a's cnum and logQ, must not alias a or b. */
int fhe_mult_relin(fhe_ctx* ctx, const fhe_ct* a, const fhe_ct* b, fhe_ct* out, void* ws, size_t ws_bytes,
                   void* stream);

/* fhe_mult_relin followed by the rescale of fhe_rescale by k bits, fused into
 * the relinearisation epilogue; out->logQ must equal a->logQ - k. */
int fhe_mult_relin_rescale(fhe_ctx* ctx, const fhe_ct* a, const fhe_ct* b, int k, fhe_ct* out, void* ws,
                           size_t ws_bytes, void* stream);

/* Batched multiply + relinearise + rescale over ciphertext pairs at
 * DIFFERENT levels of one ring (the CipherTensor batch of Sec. 6 with a
 * per-ciphertext modulus; CKKS only).  Item i has modulus 2^item_logQ[i]
 * (device int32_t[cnum], each <= logQ_max); a, b, out are device
 * uint32_t[cnum][2][L_pad][N] with L_pad >= ceil(logQ_max/32): item i's limbs
 * at and above bit item_logQ[i] must be zero on input and are zero on output.
 * Result i = fhe_mult_relin_rescale of pair i at its own level (modulus
 * 2^(item_logQ[i] - k)).  Prime counts and key rows are those of logQ_max,
 * which is exact for every item.  Workspace: FHE_OP_MULT_RAGGED at logQ_max. */
int fhe_mult_relin_rescale_ragged(fhe_ctx* ctx, const uint32_t* a, const uint32_t* b, uint32_t* out, int cnum,
                                  int L_pad, const int32_t* item_logQ, int logQ_max, int k, void* ws,
                                  size_t ws_bytes, void* stream);

/* One group of fhe_mult_relin_rescale_batch: the arguments of one
 * fhe_mult_relin_rescale_ragged call (its context fixes the ring size). */
typedef struct {
  fhe_ctx* ctx;              /* CKKS context with keys; its ring size N = 2^logN    */
  const uint32_t* a;         /* device uint32_t[cnum][2][L_pad][N]                 */
  const uint32_t* b;         /* the same shape                                     */
  uint32_t* out;             /* the same shape; must not alias a or b              */
  const int32_t* item_logQ;  /* device int32_t[cnum], each <= logQ_max             */
  int32_t cnum, L_pad, logQ_max;
  void* ws;                  /* this group's own workspace (FHE_OP_MULT_RAGGED at   */
  size_t ws_bytes;           /* logQ_max, cnum); no two groups may share bytes      */
} fhe_batch_group;

/* Schedule of the work-table transform launches (chosen by an autotuner). */
typedef struct {
  int32_t col_ctas_per_sm;   /* column stages: persistent grid of this many CTAs per SM
                                (clamped to what fits); 0: one CTA per work unit      */
  int32_t row_ctas_per_sm;   /* fused row passes: the same                             */
  int32_t col_unit_rows;     /* prime rows per column-stage work unit of the persistent
                                grid (>= 1; one CTA per unit takes 256/N1 column jobs)  */
} fhe_batch_sched;

/* Batched multiply + relinearise + rescale over pairs of SEVERAL ring sizes
 * and levels at once (the CipherTensor batching of Sec. 6, "Pairwise and
 * Broadcast Modes", across rings; CKKS only): group g is the ragged batch
 * of fhe_mult_relin_rescale_ragged with its own context, and its results are
 * exactly those of that call.  The transform stages of all groups run as
 * single launches over a work table of units (ciphertext, polynomial, prime
 * group, ring size, prime count): the forward column stages, the fused
 * transform-domain pass and the inverse column stages of the tensor
 * products, then the same three of the key switches; each group's lifts and
 * reconstructions run per group with its context's kernel forms.  Groups at
 * N <= 2^12 run their transforms per group.  1 <= ngroups <= 32, every
 * context on the current device; sched NULL = {0, 0, 1}.  Profiling of the
 * work-table launches goes to the first group's context. */
int fhe_mult_relin_rescale_batch(const fhe_batch_group* groups, int ngroups, int k, const fhe_batch_sched* sched,
                                 void* stream);

/* Rescale (rescaleBy_pairwise_into, Sec. 6): out = round(in / 2^k) mod
 * 2^(logQ - k), halves rounded up; out->logQ must equal in->logQ - k. */
int fhe_rescale(fhe_ctx* ctx, const fhe_ct* in, int k, fhe_ct* out, void* stream);

/* Modulus drop (moddownBy_pairwise_into, Sec. 6).  CKKS: out = in mod
 * 2^out->logQ, out->logQ <= in->logQ (scale unchanged).  BGV: the modulus
 * switch Q_l -> Q_{l-1} = Q_l / r, c' = (c + t [(-c) t^-1]_r) / r (centred),
 * out->level = in->level - 1, no aliasing. */
int fhe_moddown(fhe_ctx* ctx, const fhe_ct* in, fhe_ct* out, void* stream);

/* Left rotation by `step` slots (leftrotate_broadcast_into, Sec. 6; negative
 * steps rotate right): kappa_g(X) = X^g, g = 5^step mod 2N, then key switching
 * with rtk_step:
 *   out = (kappa(b), 0) + round(P^-1 kappa(a~) rtk mod P Q)  (mod Q),
 * a~ the centred representative of a (its logQ-bit two's complement, in
 * [-Q/2, Q/2)) and kappa taken over Z (coefficients negated, not reduced).
 * FHE_ENOKEY without a key for g.  out must not alias in.  Workspace:
 * FHE_OP_ROTATE (the same for one step and for fhe_rotate_hoisted). */
int fhe_rotate(fhe_ctx* ctx, const fhe_ct* in, int step, fhe_ct* out, void* ws, size_t ws_bytes, void* stream);

/* The rotations of one ciphertext batch by nsteps steps (1..4096) at once:
 * outs[s] (host array of nsteps ciphertext descriptors, device data) receives
 * fhe_rotate(in, steps[s]), bit for bit.  The key-switch input is lifted and
 * transformed once for all steps; each automorphism is then applied as a
 * permutation of the transform (hoisted rotations).  Outputs must not alias
 * the input or each other. */
int fhe_rotate_hoisted(fhe_ctx* ctx, const fhe_ct* in, const int* steps, int nsteps, fhe_ct* const* outs, void* ws,
                       size_t ws_bytes, void* stream);

/* Complex conjugation of the slots (conjugate_pairwise_into, Sec. 6): the
 * automorphism X -> X^(2N-1) with key switching by the conjugation key, in the
 * form of fhe_rotate.  FHE_ENOKEY without a conjugation key (fhe_keygen makes
 * one; fhe_keygen_conjugation injects one).  Workspace: FHE_OP_ROTATE. */
int fhe_conjugate(fhe_ctx* ctx, const fhe_ct* in, fhe_ct* out, void* ws, size_t ws_bytes, void* stream);

/* Limb-domain operations (Sec. 5: add, subtract, negate without RNS).  For
 * fhe_add / fhe_sub (CKKS), b->cnum may be 1 (broadcast mode: b is added to or
 * subtracted from every ciphertext of a; out must not alias b). */
int fhe_add(fhe_ctx* ctx, const fhe_ct* a, const fhe_ct* b, fhe_ct* out, void* stream);
int fhe_sub(fhe_ctx* ctx, const fhe_ct* a, const fhe_ct* b, fhe_ct* out, void* stream);
int fhe_negate(fhe_ctx* ctx, const fhe_ct* in, fhe_ct* out, void* stream);
/* Multiply by a signed integer constant c, |c| < 2^31 (multconst with an
 * integer-encoded scalar). */
int fhe_mult_const(fhe_ctx* ctx, const fhe_ct* in, int32_t c, fhe_ct* out, void* stream);

/* Add an integer constant (addconst, Sec. 6): coefficient 0 of b gains
 * value * 2^shift (mod 2^logQ), i.e. every slot gains value 2^shift / Delta.
 * CKKS only; 0 <= shift < logQ; out may alias in. */
int fhe_add_const(fhe_ctx* ctx, const fhe_ct* in, int64_t value, int shift, fhe_ct* out, void* stream);

/* addconst_pairwise_into (Sec. 6): ciphertext c gains values[c] * 2^shift at
 * coefficient 0 of b (values: device int64_t[cnum]).  CKKS only; out may alias in. */
int fhe_add_const_vec(fhe_ctx* ctx, const fhe_ct* in, const int64_t* values, int shift, fhe_ct* out, void* stream);

/* imult_pairwise_into (Sec. 6): multiplication of every slot by the imaginary
 * unit, i.e. of both polynomials by X^(N/2) (X^(N/2) evaluates to i at every
 * slot's root 5^j, 5^j = 1 mod 4): coefficient j moves to j + N/2 and is
 * negated when it wraps past X^N = -1.  No key and no noise growth.  CKKS
 * only; out must not alias in. */
int fhe_imult(fhe_ctx* ctx, const fhe_ct* in, fhe_ct* out, void* stream);

/* multconstvec_pairwise_into (Sec. 6): multiplication by encoded plaintext
 * polynomials, out = (b m, a m) mod 2^logQ.  pt: device uint32_t[pt_cnum][L][N],
 * each coefficient m mod 2^logQ (two's complement for negative values);
 * pt_cnum = cnum pairs plaintext c with ciphertext c, pt_cnum = 1 broadcasts
 * one plaintext (multconst_broadcast_into with a vector constant).  The
 * product is exact in Z[X]/(X^N + 1) before the reduction (one ring product
 * of each polynomial, Sec. 5 pipeline).  out->log_scale = in's + pt_log_scale
 * (follow with fhe_rescale).  CKKS only; out must not alias in.
 * Workspace: FHE_OP_MULT_PLAIN. */
int fhe_mult_plain(fhe_ctx* ctx, const fhe_ct* in, const uint32_t* pt, int pt_cnum, double pt_log_scale, fhe_ct* out,
                   void* ws, size_t ws_bytes, void* stream);

/* The big-integer negacyclic multiplier of Sec. 5 on its own:
 *   out = a * b mod 2^logOut in Z[X]/(X^N + 1),
 * a: device uint32_t[cnum][La][N], b: device uint32_t[cnum][Lb][N] (unsigned
 * canonical limbs), out: device uint32_t[cnum][ceil(logOut/32)][N].
 * logOut <= 32 (La + Lb) + logN + 1 gives the exact product. */
int fhe_ring_mul(fhe_ctx* ctx, const uint32_t* a, int La, const uint32_t* b, int Lb, int logOut, uint32_t* out,
                 int cnum, void* ws, size_t ws_bytes, void* stream);

/* fhe_mult_relin_rescale for callers that cannot allocate device memory.
 * The paper has no counterpart; this exists for the library's users.
 * Some callers cannot call cudaMalloc (or any allocator) where they multiply:
 * hosts that forbid allocation after start-up (real-time or embedded
 * services, where an allocation may block or fail at a bad moment), and
 * plug-ins of other runtimes that must not touch the process's device
 * allocator (it belongs to the host runtime).  This call takes no
 * workspace and allocates nothing (no cudaMalloc/cudaFree, no allocator
 * callback).  Its scratch is one static device array of 32 MiB that every GPU
 * loading the library holds until the process exits; a call whose scratch
 * need (fhe_workspace_bytes(ctx, FHE_OP_MULT, a->logQ, a->cnum)) exceeds
 * 32 MiB is rejected with FHE_EINVAL before anything is enqueued, as are a
 * BGV context and k < 1 (as for fhe_mult_relin_rescale).  The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress)
 * with the context's device current; make that first call before any stream
 * capture.  All calls share the one array and it keeps the last call's
 * contents (every region is written before it is read, so nothing needs
 * clearing).  Calls whose GPU work overlaps, for example calls on two streams
 * of one process, use the same array at the same time: they race and give
 * wrong results, so issue them on one stream (each process has its own
 * array).  Arguments and results are as for fhe_mult_relin_rescale. */
int fhe_mult_relin_rescale_noalloc(fhe_ctx* ctx, const fhe_ct* a, const fhe_ct* b, int k, fhe_ct* out,
                                   void* stream);

/* Kernel forms of the context's later calls (a schedule an autotuner picks;
 * no counterpart in the paper): the reconstruction `crt` (FHE_CRT_*, as at
 * creation), the lift `lift` and the transform schedule of ring products
 * `ntt`.  Every combination gives bit-identical results.  Applies to work
 * enqueued after the call (a CUDA graph keeps the forms it was captured
 * with); not thread-safe with concurrent calls on the same context. */
#define FHE_LIFT_AUTO 0  /* tensor cores when crt is FHE_CRT_DIRECT / _CVT, integer otherwise */
#define FHE_LIFT_INT 1   /* 24-bit-digit / 96-bit-accumulator integer lift                    */
#define FHE_LIFT_TC 2    /* tcgen05 byte-digit GEMM where it applies (L < 64, r <= 128)        */
#define FHE_NTT_FUSED 0  /* N > 2^12: column pass, one fused row pass (forward rows, products,
                            inverse rows), column pass                                        */
#define FHE_NTT_SPLIT 1  /* full forward transforms, pointwise products, full inverse transforms */
#define FHE_NTT_FUSED_GROUPS 2 /* the fused row pass of the tensor product with one operand row per
                                  16-thread group (smaller per-thread code), products through
                                  shared memory                                                 */
int fhe_set_forms(fhe_ctx* ctx, int crt, int lift, int ntt);

/* Diagnostics (no counterpart in the paper; measurement support).
 * Kernel classes: */
#define FHE_K_LIFT 0      /* limb -> RNS lift                        */
#define FHE_K_NTT_FWD 1   /* forward NTT passes                      */
#define FHE_K_NTT_INV 2   /* inverse NTT passes                      */
#define FHE_K_POINTWISE 3 /* transform-domain products               */
#define FHE_K_CRT 4       /* Garner reconstruction + fused epilogue  */
#define FHE_K_LIMB 5      /* limb-domain kernels (rescale, ...)      */
#define FHE_K_NTT_PW 6    /* fused transform-domain pass: forward row
                             stages, pointwise products, inverse row
                             stages of a ring product                */
#define FHE_K_COUNT 7
/* Reset the per-class counters of `ctx`; with enable != 0, also bracket
 * every subsequent launch with CUDA events on its stream (adds two event
 * records per launch).  Not thread-safe with concurrent calls on ctx. */
int fhe_profile_reset(fhe_ctx* ctx, int enable);
/* Kernels launched in class `kclass` since the last reset, and (when timing
 * was enabled) the summed event-measured device time in milliseconds.
 * Synchronises on the recorded events.  FHE_EINVAL for a bad class. */
int fhe_profile_read(fhe_ctx* ctx, int kclass, int64_t* launches, double* ms);

/* CKKS encoding on the GPU (Sec. 2 "Fast Fourier Transform"; HEAAN slots):
 * z: device complex double [cnum][N/2] (real, imaginary interleaved), full
 * packing; pt: device uint32_t[cnum][ceil(logQ/32)][N] receives m with
 * m(zeta^(5^j)) ~= 2^log_scale z_j, zeta = exp(i pi / N), i.e. the integer
 * nearest (ties to even) to the inverse canonical embedding, as logQ-bit two's
 * complement.  Requires 2^log_scale max|z_j| < 2^61 (0 <= log_scale <= 62).
 * Double-precision DFTs: coefficients can differ by one from another
 * implementation's rounding where the exact value lies within about 2^-40 of a
 * half-integer.  Workspace: FHE_OP_ENCODE (cnum). */
int fhe_ckks_encode(fhe_ctx* ctx, const double* z, int cnum, int log_scale, int logQ, uint32_t* pt, void* ws,
                    size_t ws_bytes, void* stream);

/* CKKS decoding on the GPU: pt device uint32_t[cnum][ceil(logQ/32)][N] holding
 * signed plaintexts in two's complement (as fhe_decrypt writes them);
 * z: device complex double [cnum][N/2] receives m(zeta^(5^j)) / 2^log_scale.
 * Workspace: FHE_OP_ENCODE (cnum). */
int fhe_ckks_decode(fhe_ctx* ctx, const uint32_t* pt, int cnum, int logQ, double log_scale, double* z, void* ws,
                    size_t ws_bytes, void* stream);

/* BGV slot batching (Sec. 2 "Chinese Remainder Theorem", polynomial CRT):
 * for a prime t = 1 (mod 2N) (N <= 2^15), slot k of a plaintext m in
 * Z_t[X]/(X^N + 1) is m(psi^(2k+1)) mod t, psi = g^((t-1)/(2N)) with g the
 * smallest primitive root mod t; slot-wise products are ring products.
 * fhe_bgv_encode: slots device uint32_t[cnum][N] (values mod t) -> the
 * coefficients of m in [0, t), ciphertext c's at pt + c * pt_stride (pass
 * L N to write limb 0 of an fhe_encrypt input whose other limbs are zero).
 * fhe_bgv_decode: the inverse, from coefficients at pt + c * pt_stride (as
 * fhe_decrypt writes them for BGV: pt_stride = N).  FHE_EINVAL when t is not
 * such a prime. */
int fhe_bgv_encode(fhe_ctx* ctx, const uint32_t* slots, int cnum, uint32_t* pt, size_t pt_stride, void* stream);
int fhe_bgv_decode(fhe_ctx* ctx, const uint32_t* pt, size_t pt_stride, int cnum, uint32_t* slots, void* stream);

/* Self-test of failure detection (no counterpart in the paper): launches one
 * thread that waits on a shared-memory barrier nothing arrives on, polling at
 * most `tries` (1..100000) times with a 1 us suspend hint, then records the
 * timeout in the device status word and returns, exactly as a pipeline wait of
 * the tensor-core kernels does when it gives up.  The next fhe_sync returns
 * FHE_ETIMEOUT (and clears the word); the context stays usable. */
int fhe_selftest_wait_timeout(int tries, void* stream);

/* Number of NTT primes the library uses for a ring product whose exact
 * result is bounded by 2^bound_bits in absolute value (one spare prime for
 * the sign, Sec. 5 signed handling).  Informational. */
int fhe_primes_for_bound(int bound_bits);

#ifdef __cplusplus
}
#endif

#endif /* FHE_GB300_H */
