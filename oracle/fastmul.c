/*
 * Test oracle (infrastructure, not product): exact negacyclic product of two
 * polynomials with big-integer coefficients, for ring sizes where the
 * pure-Python schoolbook product (Sec. 2, Eq. schoolbook and Eq. reduction)
 * is too slow.
 *
 * What it computes is the plain definition
 *     c_i = sum_{j+k=i} a_j b_k - sum_{j+k=i+N} a_j b_k      (over Z)
 * and it returns c_i modulo 2^(32*Lout) as two's-complement limbs.  When
 * Lout is wide enough for the bound N*|a|max*|b|max this is c_i exactly.
 *
 * How, chosen to share nothing with the CUDA path (which works with 30/31-bit
 * primes, Shoup/Montgomery-32 arithmetic and Garner's mixed radix form):
 *   - 62-bit primes p = 1 (mod 2^17), 64-bit Montgomery multiplication;
 *   - per prime: twist by psi^j, textbook iterative radix-2 cyclic NTT with
 *     omega = psi^2 and explicit bit reversal, pointwise product, inverse,
 *     untwist, times N^-1 (Eq. ntt_mul with Eq. negacyclic_ntt/intt);
 *   - the plain CRT sum of Eq. crt_composition evaluated in full
 *     multi-precision, reduced into [0, M) by repeated subtraction and then
 *     centred (x > M/2 -> x - M), M > 2*bound.
 * Single-threaded and untuned on purpose.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

/* ---------------------------------------------------------------- primes */

static uint64_t mulmod_slow(uint64_t a, uint64_t b, uint64_t p) { return (uint64_t)(((u128)a * b) % p); }

static uint64_t powmod_slow(uint64_t a, uint64_t e, uint64_t p) {
  uint64_t r = 1 % p;
  a %= p;
  while (e) {
    if (e & 1) r = mulmod_slow(r, a, p);
    a = mulmod_slow(a, a, p);
    e >>= 1;
  }
  return r;
}

/* Deterministic Miller-Rabin for n < 3.3e24 (bases 2..37). */
static int is_prime_u64(uint64_t n) {
  static const uint64_t bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  if (n < 2) return 0;
  for (int i = 0; i < 12; ++i) {
    if (n % bases[i] == 0) return n == bases[i];
  }
  uint64_t d = n - 1;
  int s = 0;
  while ((d & 1) == 0) { d >>= 1; ++s; }
  for (int i = 0; i < 12; ++i) {
    uint64_t x = powmod_slow(bases[i], d, n);
    if (x == 1 || x == n - 1) continue;
    int comp = 1;
    for (int r = 1; r < s; ++r) {
      x = mulmod_slow(x, x, n);
      if (x == n - 1) { comp = 0; break; }
    }
    if (comp) return 0;
  }
  return 1;
}

#define ORACLE_MAX_PRIMES 256
static uint64_t g_primes[ORACLE_MAX_PRIMES];
static int g_nprimes = 0;

/* Primes p < 2^62 with p = 1 (mod 2^17), largest first. */
static void ensure_primes(int k) {
  if (g_nprimes >= k) return;
  uint64_t step = (uint64_t)1 << 17;
  uint64_t c = (g_nprimes == 0) ? ((((uint64_t)1 << 62) / step) * step + 1) : g_primes[g_nprimes - 1];
  if (c > ((uint64_t)1 << 62)) c -= step;
  while (g_nprimes < k) {
    c -= step;
    if (is_prime_u64(c)) g_primes[g_nprimes++] = c;
  }
}

/* ----------------------------------------------------- 64-bit Montgomery */

typedef struct {
  uint64_t p, pinv_neg, r2; /* pinv_neg = -p^-1 mod 2^64, r2 = 2^128 mod p */
} mont_t;

static mont_t mont_make(uint64_t p) {
  mont_t m;
  m.p = p;
  uint64_t inv = 1; /* Newton iteration for p^-1 mod 2^64 */
  for (int i = 0; i < 7; ++i) inv *= 2 - p * inv;
  m.pinv_neg = (uint64_t)0 - inv;
  uint64_t r1 = (uint64_t)(((u128)1 << 64) % p);
  m.r2 = mulmod_slow(r1, r1, p);
  return m;
}

/* a*b*2^-64 mod p for a, b < p < 2^62 */
static inline uint64_t mont_mul(const mont_t* m, uint64_t a, uint64_t b) {
  u128 t = (u128)a * b;
  uint64_t u = (uint64_t)t * m->pinv_neg;
  u128 s = t + (u128)u * m->p;
  uint64_t r = (uint64_t)(s >> 64);
  return r >= m->p ? r - m->p : r;
}
static inline uint64_t to_mont(const mont_t* m, uint64_t a) { return mont_mul(m, a, m->r2); }
static inline uint64_t from_mont(const mont_t* m, uint64_t a) { return mont_mul(m, a, 1); }

/* ---------------------------------------------------- cyclic NTT, length n */

static unsigned bitrev(unsigned x, int bits) {
  unsigned r = 0;
  for (int i = 0; i < bits; ++i) { r = (r << 1) | (x & 1); x >>= 1; }
  return r;
}

/* In place, values in Montgomery form; w = primitive n-th root (Montgomery form). */
static void ntt_cyclic(const mont_t* m, uint64_t* a, int logn, uint64_t w) {
  unsigned n = 1u << logn;
  for (unsigned i = 0; i < n; ++i) {
    unsigned j = bitrev(i, logn);
    if (j > i) { uint64_t t = a[i]; a[i] = a[j]; a[j] = t; }
  }
  for (unsigned len = 2; len <= n; len <<= 1) {
    uint64_t wl = w; /* w^(n/len) */
    for (unsigned s = len; s < n; s <<= 1) wl = mont_mul(m, wl, wl);
    for (unsigned i = 0; i < n; i += len) {
      uint64_t x = to_mont(m, 1);
      for (unsigned j = 0; j < len / 2; ++j) {
        uint64_t u = a[i + j];
        uint64_t v = mont_mul(m, a[i + j + len / 2], x);
        uint64_t s1 = u + v; if (s1 >= m->p) s1 -= m->p;
        uint64_t d1 = u >= v ? u - v : u + m->p - v;
        a[i + j] = s1;
        a[i + j + len / 2] = d1;
        x = mont_mul(m, x, wl);
      }
    }
  }
}

/* ------------------------------------------------------ big-integer helpers */

/* little-endian u64 limbs */
static void big_mul_small(uint64_t* x, int n, uint64_t s) {
  u128 carry = 0;
  for (int i = 0; i < n; ++i) {
    u128 t = (u128)x[i] * s + carry;
    x[i] = (uint64_t)t;
    carry = t >> 64;
  }
}
static int big_cmp(const uint64_t* a, const uint64_t* b, int n) {
  for (int i = n - 1; i >= 0; --i) {
    if (a[i] != b[i]) return a[i] > b[i] ? 1 : -1;
  }
  return 0;
}
static void big_sub(uint64_t* a, const uint64_t* b, int n) { /* a -= b, a >= b */
  uint64_t borrow = 0;
  for (int i = 0; i < n; ++i) {
    uint64_t bi = b[i];
    uint64_t d = a[i] - bi - borrow;
    borrow = (a[i] < bi) || (a[i] - bi < borrow);
    a[i] = d;
  }
}

/* ------------------------------------------------------------- the product */

/* residue of a two's-complement limb number mod p */
static uint64_t limbs_mod(const uint32_t* x, int L, size_t stride, int is_signed, uint64_t p, const uint64_t* pw) {
  u128 acc = 0; /* sum limb_l * (2^(32 l) mod p): each term < 2^94, L <= 2^30 terms fit */
  for (int l = 0; l < L; ++l) acc += (u128)x[(size_t)l * stride] * pw[l];
  uint64_t r = (uint64_t)(acc % p);
  if (is_signed && (x[(size_t)(L - 1) * stride] >> 31)) { /* value - 2^(32L) */
    uint64_t t = pw[L];
    r = r >= t ? r - t : r + p - t;
  }
  return r;
}

/*
 * out[l*N + i] (l < Lout) = limb l of c_i mod 2^(32 Lout), two's complement.
 * a: La limbs x N (limb-major, N contiguous); b likewise.  a_signed/b_signed:
 * the top bit of the top limb is a sign bit.  bound_bits: an upper bound on
 * log2 |c_i| (the caller passes logN + bits(a) + bits(b)).
 * Returns 0 on success, negative on bad arguments or allocation failure.
 */
int oracle_negacyclic_mul(int logN, const uint32_t* a, int La, int a_signed, const uint32_t* b, int Lb,
                          int b_signed, uint32_t* out, int Lout, int bound_bits) {
  if (logN < 0 || logN > 16 || La < 1 || Lb < 1 || Lout < 1 || bound_bits < 1) return -1;
  const int N = 1 << logN;
  /* k primes of > 61.99 bits each with product > 2^(bound_bits + 2) */
  int k = (bound_bits + 2) / 61 + 1;
  if (k > ORACLE_MAX_PRIMES) return -2;
  ensure_primes(k);
  const int Lmax = (La > Lb ? La : Lb) + 1;

  uint64_t* res = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)k * N); /* residues of c, prime-major */
  uint64_t* fa = (uint64_t*)malloc(sizeof(uint64_t) * N);
  uint64_t* fb = (uint64_t*)malloc(sizeof(uint64_t) * N);
  uint64_t* pw = (uint64_t*)malloc(sizeof(uint64_t) * (Lmax + 1));
  if (!res || !fa || !fb || !pw) { free(res); free(fa); free(fb); free(pw); return -3; }

  for (int pi = 0; pi < k; ++pi) {
    const uint64_t p = g_primes[pi];
    mont_t m = mont_make(p);
    for (int l = 0; l <= Lmax; ++l) pw[l] = powmod_slow(2, 32ull * (uint64_t)l, p);
    /* psi: primitive 2N-th root of unity */
    uint64_t psi = 0;
    for (uint64_t x = 2;; ++x) {
      uint64_t cand = powmod_slow(x, (p - 1) / (2ull * (uint64_t)N), p);
      if (powmod_slow(cand, (uint64_t)N, p) == p - 1) { psi = cand; break; }
    }
    uint64_t psi_m = to_mont(&m, psi);
    uint64_t w_m = mont_mul(&m, psi_m, psi_m);
    /* twist: a_j psi^j */
    uint64_t tw = to_mont(&m, 1);
    for (int j = 0; j < N; ++j) {
      fa[j] = mont_mul(&m, to_mont(&m, limbs_mod(a + j, La, (size_t)N, a_signed, p, pw)), tw);
      fb[j] = mont_mul(&m, to_mont(&m, limbs_mod(b + j, Lb, (size_t)N, b_signed, p, pw)), tw);
      tw = mont_mul(&m, tw, psi_m);
    }
    ntt_cyclic(&m, fa, logN, w_m);
    ntt_cyclic(&m, fb, logN, w_m);
    for (int j = 0; j < N; ++j) fa[j] = mont_mul(&m, fa[j], fb[j]);
    /* inverse: NTT with omega^-1, then times N^-1 psi^-j */
    uint64_t winv = to_mont(&m, powmod_slow(mulmod_slow(psi, psi, p), p - 2, p));
    ntt_cyclic(&m, fa, logN, winv);
    uint64_t ninv = to_mont(&m, powmod_slow((uint64_t)N, p - 2, p));
    uint64_t psiinv = to_mont(&m, powmod_slow(psi, p - 2, p));
    uint64_t f = ninv;
    for (int j = 0; j < N; ++j) {
      res[(size_t)pi * N + j] = from_mont(&m, mont_mul(&m, fa[j], f));
      f = mont_mul(&m, f, psiinv);
    }
  }

  /* CRT: X = sum_i [x_i * (M/p_i)^-1]_{p_i} * (M/p_i), reduce into [0,M), centre. */
  const int W = k + 1; /* u64 limbs for values < (k+1) M */
  uint64_t* Mbig = (uint64_t*)calloc((size_t)W, sizeof(uint64_t));
  uint64_t* Mi = (uint64_t*)calloc((size_t)k * W, sizeof(uint64_t));
  uint64_t* inv = (uint64_t*)malloc(sizeof(uint64_t) * k);
  uint64_t* X = (uint64_t*)malloc(sizeof(uint64_t) * W);
  uint64_t* halfM = (uint64_t*)calloc((size_t)W, sizeof(uint64_t));
  if (!Mbig || !Mi || !inv || !X || !halfM) {
    free(res); free(fa); free(fb); free(pw); free(Mbig); free(Mi); free(inv); free(X); free(halfM);
    return -3;
  }
  Mbig[0] = 1;
  for (int i = 0; i < k; ++i) big_mul_small(Mbig, W, g_primes[i]);
  for (int i = 0; i < k; ++i) {
    uint64_t* mi = Mi + (size_t)i * W;
    mi[0] = 1;
    for (int j = 0; j < k; ++j)
      if (j != i) big_mul_small(mi, W, g_primes[j]);
    /* (M/p_i) mod p_i, then its inverse */
    u128 r = 0;
    for (int l = W - 1; l >= 0; --l) r = ((r << 64) | mi[l]) % g_primes[i];
    inv[i] = powmod_slow((uint64_t)r, g_primes[i] - 2, g_primes[i]);
  }
  for (int l = 0; l < W; ++l) halfM[l] = (Mbig[l] >> 1) | (l + 1 < W ? (Mbig[l + 1] << 63) : 0);

  for (int j = 0; j < N; ++j) {
    memset(X, 0, sizeof(uint64_t) * W);
    for (int i = 0; i < k; ++i) {
      uint64_t y = mulmod_slow(res[(size_t)i * N + j], inv[i], g_primes[i]);
      const uint64_t* mi = Mi + (size_t)i * W;
      u128 carry = 0;
      for (int l = 0; l < W; ++l) {
        u128 t = (u128)mi[l] * y + X[l] + carry;
        X[l] = (uint64_t)t;
        carry = t >> 64;
      }
    }
    while (big_cmp(X, Mbig, W) >= 0) big_sub(X, Mbig, W);
    int negative = big_cmp(X, halfM, W) > 0; /* X > M/2 (M odd) */
    if (negative) { /* X <- M - X, magnitude of the negative result */
      uint64_t* t = (uint64_t*)malloc(sizeof(uint64_t) * W);
      memcpy(t, Mbig, sizeof(uint64_t) * W);
      big_sub(t, X, W);
      memcpy(X, t, sizeof(uint64_t) * W);
      free(t);
    }
    /* emit |c| or -|c| as 32-bit two's complement limbs */
    uint32_t borrow = 1;
    for (int l = 0; l < Lout; ++l) {
      uint32_t limb = 0;
      int w64 = l / 2;
      if (w64 < W) limb = (uint32_t)(X[w64] >> (32 * (l & 1)));
      if (negative) {
        uint64_t v = (uint64_t)(uint32_t)~limb + borrow;
        limb = (uint32_t)v;
        borrow = (uint32_t)(v >> 32);
      }
      out[(size_t)l * N + j] = limb;
    }
  }
  free(res); free(fa); free(fb); free(pw); free(Mbig); free(Mi); free(inv); free(X); free(halfM);
  return 0;
}
