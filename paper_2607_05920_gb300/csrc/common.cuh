// Internal declarations of libfhe_gb300: the context, the modular arithmetic
// used by every kernel, and the kernel launchers shared between translation
// units.  Nothing here is part of the public C ABI (include/fhe.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "fhe.h"

namespace fhe {

// ---------------------------------------------------------------- limits
constexpr int kMaxPrimes = 256;    // NTT primes available to one context
constexpr int kMaxLimbs = 128;     // widest big integer a ring product emits (4096 bits)
constexpr int kMaxLiftLimbs = 128; // widest operand a ring product lifts
constexpr int kLiftDigits = 64;    // 24-bit digits of the digit-lift path (operands up to 48 limbs)
constexpr int kCrtDigits = 176;    // 24-bit digit columns of the direct CRT (22 blocks of 8)
constexpr int kMaxLogN = 16;
constexpr int kMaxGaussB = 60;          // widest rounded-Gaussian support |e| <= B, B = floor(6 sigma)
constexpr double kMaxGaussSigma = 10.0;
constexpr double kDefaultSigma = 3.2;
// sampler stream tags (tag0) of the seeded key generation and encryption
constexpr uint32_t kTagSecret = 1, kTagPkA = 2, kTagPkE = 3, kTagEvA = 4, kTagEvE = 5, kTagSwA = 6, kTagSwE = 7,
                   kTagEncV = 8;

// Thresholds of the rounded-Gaussian sampler (see sampler.cu).
struct GaussTable {
  uint32_t thr[2 * kMaxGaussB];
  int B = 0;
};

// Error reporting (thread-local message, see fhe_last_error).
void set_error(const char* fmt, ...);
#define FHE_CHECK_CUDA(expr)                                                     \
  do {                                                                           \
    cudaError_t _e = (expr);                                                     \
    if (_e != cudaSuccess) {                                                     \
      ::fhe::set_error("%s:%d: %s: %s", __FILE__, __LINE__, #expr,               \
                       cudaGetErrorString(_e));                                  \
      return FHE_ECUDA;                                                          \
    }                                                                            \
  } while (0)

// ------------------------------------------------------------ the context
// A switching key (relinearisation or rotation) in NTT form over the first
// `rows` primes: uint32_t[2][rows][N] (b' rows, then a' rows).
struct SwitchKey {
  uint32_t* ntt = nullptr;
  int rows = 0;
};

struct BgvLevel;
struct BgvConsts;

// Per-kernel-class launch counters and optional CUDA-event timing.
struct Profile {
  int64_t launches[FHE_K_COUNT] = {};
  bool timing = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[FHE_K_COUNT];
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get_event();
  void reset(bool enable);
  ~Profile();
};

// Brackets the kernel launches of one launcher call (kernels: how many).
class ProfScope {
 public:
  ProfScope(const fhe_ctx* ctx, int kclass, int kernels, cudaStream_t st);
  ~ProfScope();

 private:
  Profile* p_;
  int k_;
  cudaStream_t st_;
  cudaEvent_t stop_ = nullptr;
};

}  // namespace fhe

struct fhe_ctx {
  fhe_params prm{};
  int N = 0;
  int device = 0;
  fhe_alloc_fn alloc = nullptr;
  fhe_free_fn free_ = nullptr;
  void* alloc_user = nullptr;

  // primes (host copy) and how many the tables cover
  int R = 0;
  std::vector<uint32_t> q;

  // device tables (Sec. 5 "Precomputation")
  uint32_t* d_q = nullptr;        // [R]
  uint32_t* d_qinv = nullptr;     // [R]  q^-1 mod 2^32 (Montgomery)
  uint2* d_psi2 = nullptr;        // [R][N] (psi^brv(k), floor(w 2^32 / q)): forward twiddles (bit-reversed
                                  // order) with their Shoup companions, one 64-bit load per butterfly
  uint2* d_ipsi2 = nullptr;       // [R][N] (psi^-brv(k), Shoup companion)
  uint32_t* d_nscale = nullptr;   // [R]  N^-1 * 2^32 mod q (INTT scale, undoes one Montgomery factor;
                                  // applied in the reconstruction)
  uint32_t* d_nscale_sh = nullptr;// [R]
  uint32_t* d_pow2 = nullptr;     // [R][kMaxLiftLimbs] 2^(32 l) mod q
  uint32_t* d_pow24 = nullptr;    // [R][kLiftDigits] 2^(24 m) mod q
  uint32_t* d_red = nullptr;      // [R][4] {2^32 mod q, shoup, 2^64 mod q, shoup}
  uint2* d_garner = nullptr;      // [R][R] at [k*R + j] = {[q_j^-1]_{q_k}, shoup}, j < k
  uint32_t* d_mprod = nullptr;    // [R+1][kMaxLimbs] prod_{i<k} q_i mod 2^(32 kMaxLimbs)
  // direct CRT over the first r primes, for every r in [1, R]; rows of set r start at r(r-1)/2
  uint32_t* d_crt_qhat = nullptr; // [R(R+1)/2][kMaxLimbs] (M_r / q_i) mod 2^(32 kMaxLimbs)
  uint2* d_crt_inv = nullptr;     // [R(R+1)/2] {[(M_r / q_i)^-1 N^-1 2^32]_{q_i}, shoup}
  uint32_t* d_crt_negm = nullptr; // [R+1][kMaxLimbs] (-M_r) mod 2^(32 kMaxLimbs)
  float* d_invq = nullptr;        // [R] 1/q_i rounded to fp32
  uint32_t* d_crt_dig = nullptr;  // per r: [r+1][kCrtDigits] 24-bit digits of (M_r/q_i) mod 2^4096, last row -M_r
  // the same dense product on the tcgen05 tensor cores: per r, the B operand [P][K] in f16, the
  // balanced byte digits of (M_r/q_i) and -M_r Toeplitz-shifted by the digit index a of y_i
  // (B[p][4i + a] = c_{i,p-a}); K in chunks of 64, each chunk [p/8][k/8][p%8][k%8] (K-major core
  // matrices, no swizzle) for p < 16 crt_tc_mt; set r starts at crt_tc_off[r] (f16 elements)
  uint16_t* d_crt_tc = nullptr;
  // tensor-core lift: B operand [4R rows (i, a)][4 kMaxLiftLimbs k] f16 in K-major core-matrix order
  // [row/8][k/8][row%8][k%8], digit a of (2^(8k) 2^32 mod q_i) (digits 0..2 balanced, 3 in [0, 128]);
  // and per L the folded offset + 2^17 q_i, [kMaxLiftLimbs + 1][R] (see k_lift_tc)
  uint16_t* d_lift_tc = nullptr;
  uint64_t* d_lift_off = nullptr;
  uint64_t* d_lift_off_s = nullptr;  // the same offsets for the signed (two's-complement) lift
  std::vector<size_t> crt_tc_off;
  std::vector<uint8_t> crt_tc_exact22;  // per r: every column sum is below 2^22 in magnitude
  int crt_tc_mt = 0;              // output byte columns covered, in 16s
  int lift_form = 0;              // FHE_LIFT_AUTO (tensor cores with the direct CRT modes), _INT, _TC
  int ntt_form = 0;               // FHE_NTT_FUSED: ring products run their transform-domain work in one
                                  // fused row pass; FHE_NTT_SPLIT: separate transforms and products
  int crt_mode = 0;               // 0 direct CRT (tensor cores where it applies), 3 the same with cvt.rni
                                  // conversion of the column sums, 1 Garner (Eq. garner_mrc),
                                  // 2 direct CRT on the integer pipe only
  // BGV (scheme FHE_SCHEME_BGV): chain constants per level, and bit lengths of Q_l
  fhe::BgvLevel* d_bgv_levels = nullptr;
  fhe::BgvConsts* d_bgv_consts = nullptr;
  std::vector<int> bgv_bits;
  uint32_t* d_bgv_slots = nullptr;  // slot batching tables mod t (built on first use, see k_encode.cu)

  // rounded-Gaussian sampler table for params.sigma (seeded encryption and key generation)
  fhe::GaussTable gauss;

  // keys (resident)
  bool have_keys = false;
  int32_t* d_s = nullptr;          // [N] secret
  uint32_t* d_pk = nullptr;        // [2][Lq][N] public key limbs
  uint32_t* d_pk_ntt = nullptr;    // [2][r_enc][N]
  int r_enc = 0;
  uint32_t* d_s_ntt = nullptr;     // [r_dec][N]
  int r_dec = 0;
  fhe::SwitchKey evk;
  std::map<uint32_t, fhe::SwitchKey> rtk;  // by Galois element g

  // diagnostics
  mutable fhe::Profile prof;

  // every allocation the context owns, for destroy
  std::vector<std::pair<void*, size_t>> owned;
};

namespace fhe {

// --------------------------------------------------------- host utilities
int primes_for_bound(const fhe_ctx* ctx, int bound_bits);  // uses ctx->q
int primes_for_bound_global(int bound_bits);
const std::vector<uint32_t>& global_primes();
void* ctx_alloc(fhe_ctx* ctx, size_t bytes);
void ctx_free(fhe_ctx* ctx, void* p);
int build_tables(fhe_ctx* ctx);
void free_all(fhe_ctx* ctx);
const char* last_error();

inline int limbs_for_bits(int bits) { return (bits + 31) / 32; }

// Galois element 5^step mod 2N of a left rotation by `step` slots (5 has order N/2 mod 2N;
// negative steps rotate right).
inline uint32_t galois_of_step(int N, int step) {
  const long long ord = N / 2;
  long long e = step % ord;
  if (e < 0) e += ord;
  uint64_t g = 1, b = 5, m = 2ull * N;
  while (e) {
    if (e & 1) g = g * b % m;
    b = b * b % m;
    e >>= 1;
  }
  return (uint32_t)g;
}

// --------------------------------------------------------------- sampler
// Counter-based sampler (Philox4x32-10) of sampler.cu: host draws for key generation, a kernel
// for the randomness of seeded encryption.
int gauss_table(double sigma, GaussTable* gt);
void sample_uniform_limbs(uint64_t seed, uint32_t tag0, uint32_t tag1, int n, int bits, uint32_t* out);
void sample_ternary(uint64_t seed, uint32_t tag0, uint32_t tag1, int n, int8_t* out);
void sample_sparse_ternary(uint64_t seed, uint32_t tag0, uint32_t tag1, int n, int h, int8_t* out);
void sample_gaussian(uint64_t seed, uint32_t tag0, uint32_t tag1, int n, const GaussTable& gt, int32_t* out);
// v: int8 [cnum][N], e0 / e1: int32 [cnum][N] (device)
int launch_sample_enc(const fhe_ctx* ctx, uint64_t seed, int cnum, int8_t* v, int32_t* e0, int32_t* e1,
                      cudaStream_t st);
inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// ------------------------------------------------------ device arithmetic
// All primes satisfy 2^29 < q < 2^30, so 4q < 2^32.

// a * w mod q with w's Shoup companion wp = floor(w 2^32 / q); any a < 2^32.
// Result in [0, q).  (Shoup's precomputed-quotient multiplication.)
__device__ __forceinline__ uint32_t shoup_mul(uint32_t a, uint32_t w, uint32_t wp, uint32_t q) {
  uint32_t t = __umulhi(a, wp);
  uint32_t r = a * w - t * q;  // in [0, 2q)
  return r >= q ? r - q : r;
}
// Same, result left in [0, 2q).
__device__ __forceinline__ uint32_t shoup_mul_lazy(uint32_t a, uint32_t w, uint32_t wp, uint32_t q) {
  uint32_t t = __umulhi(a, wp);
  return a * w - t * q;
}

// Montgomery product a b 2^-32 mod q for a, b < q, with qinv = q^-1 mod 2^32.
// (Montgomery 1985.)  Result in [0, q).
__device__ __forceinline__ uint32_t mont_mul(uint32_t a, uint32_t b, uint32_t q, uint32_t qinv) {
  uint32_t lo = a * b;
  uint32_t hi = __umulhi(a, b);
  uint32_t m = lo * qinv;               // m q = lo (mod 2^32)
  uint32_t mh = __umulhi(m, q);         // (a b - m q) / 2^32 = hi - mh, in (-q, q)
  uint32_t r = hi - mh;
  return (hi < mh) ? r + q : r;
}

// The same product left in (0, 2q): hi - mh + q.  Needs a b < q 2^32 (one operand may be in
// [0, 4q) when the other is in [0, q)).
__device__ __forceinline__ uint32_t mont_mul_lazy(uint32_t a, uint32_t b, uint32_t q, uint32_t qinv) {
  const uint32_t lo = a * b;
  const uint32_t hi = __umulhi(a, b);
  const uint32_t mh = __umulhi(lo * qinv, q);
  return hi - mh + q;
}

__device__ __forceinline__ uint32_t add_mod(uint32_t a, uint32_t b, uint32_t q) {
  uint32_t s = a + b;  // a, b < q < 2^30: no overflow
  return s >= q ? s - q : s;
}
__device__ __forceinline__ uint32_t sub_mod(uint32_t a, uint32_t b, uint32_t q) {
  return a >= b ? a - b : a + q - b;
}

// ------------------------------------------------------------ launchers
// Lift: residues of unsigned L-limb integers modulo primes [0, r), as representatives below 2 q
// (the tensor-core form leaves them in [0, q + 2^17); they feed forward transforms).
//   src: [npoly][L][N] (poly stride src_stride words), dst: [npoly][r][N]
//   (poly stride dst_stride words); polys of batch c at src + c*src_bstride.
int launch_lift(const fhe_ctx* ctx, const uint32_t* src, int L, size_t src_pstride, size_t src_bstride,
                uint32_t* dst, size_t dst_pstride, size_t dst_bstride, int npoly, int nbatch, int r,
                cudaStream_t st);
// The same lift of signed values: batch item b holds the two's-complement integer of
// bits(b) = item_bits ? item_bits[b] : sbits bits (bit bits(b) - 1 is the sign, limbs at and above
// bit bits(b) are ignored), i.e. the centred representative in [-2^(bits-1), 2^(bits-1)) of a value
// mod 2^bits.  L < kMaxLiftLimbs.
int launch_lift_signed(const fhe_ctx* ctx, const uint32_t* src, int L, size_t src_pstride, size_t src_bstride,
                       uint32_t* dst, size_t dst_pstride, size_t dst_bstride, int npoly, int nbatch, int r, int sbits,
                       const int32_t* item_bits, cudaStream_t st);
// Lift of small signed int32 (or int8 when is_i8) coefficients.
int launch_lift_small(const fhe_ctx* ctx, const void* src, bool is_i8, size_t src_bstride, uint32_t* dst,
                      size_t dst_bstride, int nbatch, int r, cudaStream_t st);

// In-place negacyclic NTT / INTT on `rows` rows of N words; row k uses prime
// (k % r) -- rows are grouped [..][r][N].  The inverse leaves its result in
// [0, 2q) without the scale N^-1 2^32 (which also undoes one Montgomery
// factor): the reconstruction's constants (d_crt_inv) and Garner's first step
// apply it, so an inverse transform must be followed by launch_garner.
//  rows are taken in `ngroups` groups of `group_rows` consecutive rows, group g
//  starting at row g * group_stride; within a group, row k uses prime k % r.
int launch_ntt(const fhe_ctx* ctx, uint32_t* data, int ngroups, int group_rows, int group_stride, int r,
               bool inverse, cudaStream_t st);

// Pointwise products in the transform domain (Montgomery; Sec. 5 element-wise
// arithmetic, Karatsuba of Sec. 5 for the tensor).
//  tensor: X = [nbatch][4][r][N] holding (B1, A1, B2, A2) -> (D0, D1, D2) in rows 0..3r
int launch_pointwise_tensor(const fhe_ctx* ctx, uint32_t* X, int r, int nbatch, cudaStream_t st);
// Ring products in the transform domain, fused (forward transforms, pointwise products, inverse transforms):
//  tensor: X = [nbatch][4][r][N] (B1, A1, B2, A2) -> D0, D1, D2 (coefficient form) in blocks 0..2
//  key:    Y = [nbatch][2][r][N] block 0 (D) -> D K_b in block 0, D K_a in block 1, K = [2][krows][N]
int launch_ring_tensor(const fhe_ctx* ctx, uint32_t* X, int r, int nbatch, cudaStream_t st);
int launch_ring_key(const fhe_ctx* ctx, uint32_t* Y, const uint32_t* K, int krows, int r, int nbatch,
                    cudaStream_t st);
// Key switch of an automorphism kappa_g (rotation, conjugation) from the forward transform of its
// input: AH = [nbatch][r][N] (transform form, fully reduced), K = [2][krows][N]; writes
// Y = [nbatch][2][r][N] = the coefficient-form products kappa_g(a) K_b, kappa_g(a) K_a (one
// Montgomery factor removed by the inverse transform's scale, as in launch_ring_key).
int launch_key_perm(const fhe_ctx* ctx, const uint32_t* AH, uint32_t* Y, const uint32_t* K, int krows, int r,
                    int nbatch, uint32_t g, cudaStream_t st);

// Work table of one transform stage over many ring products at once (several ring sizes
// N >= 2^13 and prime counts): one segment per group of ring products, with that group's buffer,
// tables and shape.  The table travels by value in the launch's parameter block, so a captured
// graph holds it.  The launcher numbers the work units of every segment:
//  column stages, persistent grid: a unit is `unit_rows` consecutive rows of the row map
//    (consecutive primes of one polynomial), all 256 columns; one CTA per unit: a unit is one
//    round of 256 / N1 column jobs (32 columns of one row each); rows are independent;
//  fused row passes: a unit is one block of 8 matrix rows of one (ciphertext, prime).
constexpr int kTableSegs = 32;
struct NttSeg {
  uint32_t* data;         // the group's ring-product buffer (X or Y of the fused launchers)
  const uint32_t* key;    // key pass: switching key rows [2][krows][N] in transform form
  const uint2* tw;        // forward twiddle pairs of this ring
  const uint2* itw;       // inverse twiddle pairs
  const uint32_t* q;      // primes
  const uint32_t* qinv;   // q^-1 mod 2^32
  int group_rows, group_stride;  // column stages: the row map of launch_ntt
  int r, logN, nb, krows; // primes, log ring size, ciphertexts, key rows
  int rows;               // column stages: rows of the row map
  int units, unit0;       // set by the launcher
};
struct NttTable {
  int nseg, total, unit_rows;
  NttSeg seg[kTableSegs];
};
enum TableStage { kTableColsFwd = 0, kTableColsInv = 1, kTableRowsTensor = 2, kTableRowsKey = 3 };
// Launches one stage over the table (every segment at logN >= 13).  ctas_per_sm > 0: a persistent
// grid of that many CTAs per SM (clamped to what fits) walking the units in strides; 0: one CTA
// per unit.
int launch_ntt_table(const fhe_ctx* prof_ctx, NttTable& t, int stage, int ctas_per_sm, cudaStream_t st);
//  key: Y = [nbatch][2][r][N]; row block 0 holds D (in), outputs D*K_b into block 0 and
//  D*K_a into block 1 with K = [2][krows][N] (first r rows used).
int launch_pointwise_key(const fhe_ctx* ctx, uint32_t* Y, const uint32_t* K, int krows, int r, int nbatch,
                         cudaStream_t st);
//  Z at batch stride z_bstride (the plain form: r N)
int launch_pointwise_mul_strided(const fhe_ctx* ctx, uint32_t* Z, size_t z_bstride, const uint32_t* A,
                                 size_t a_bstride, const uint32_t* B, size_t b_bstride, int r, int nbatch,
                                 cudaStream_t st);
//  general: Z[b][k][n] = A[b][k][n] * B[(b*bstride_b)][k][n]  (bstride_b 0 = broadcast)
int launch_pointwise_mul(const fhe_ctx* ctx, uint32_t* Z, const uint32_t* A, size_t a_bstride, const uint32_t* B,
                         size_t b_bstride, int r, int nbatch, cudaStream_t st);

// Garner reconstruction (Sec. 2 Eq. garner_mrc; Sec. 5 RNS-to-limb) of r
// residue rows into limbs, with a fused epilogue.
enum class Epi : int {
  kStore = 0,     // out = X mod 2^out_bits
  kRelin = 1,     // out = (add + round(X / 2^shift)) mod 2^out_bits, then optional rescale by k2
  kAddSmall = 2,  // out = (X + add + small) mod 2^out_bits, add/small optional; negate X first if neg
  kDecrypt = 3,   // out = centred (X + add) mod 2^out_bits, sign-extended to out limbs
};
struct EpiArgs {
  Epi kind = Epi::kStore;
  int out_bits = 0;          // modulus 2^out_bits of the result
  const int32_t* item_bits = nullptr;  // if set: per batch item modulus bits (overrides out_bits)
  int out_limbs = 0;         // limbs written per coefficient
  const uint32_t* add = nullptr;  // limbs [L_add][N] per poly (batch stride add_bstride)
  int add_limbs = 0;
  size_t add_pstride = 0;    // between polys
  size_t add_bstride = 0;
  int add_polys = 1 << 30;   // only polys with index < add_polys receive `add`
  const int32_t* small = nullptr;  // int32 [N] per batch for poly 0 (batch stride small_bstride)
  const int32_t* small1 = nullptr; // int32 [N] per batch for poly 1
  size_t small_bstride = 0;
  int shift = 0;             // kRelin: log P
  int k2 = 0;                // kRelin: extra rescale bits (0 = none)
  int negate = 0;            // kAddSmall: use -X
};
// in: [nbatch][npoly][r][N] (poly stride in_pstride, batch in_bstride);
// out: [nbatch][npoly][out_limbs][N] (strides out_pstride, out_bstride).
unsigned int read_dev_status();   // nonzero (then cleared) after a bounded device wait gave up
unsigned int read_lift_status();  // the same for the lift kernels
int launch_garner(const fhe_ctx* ctx, const uint32_t* in, size_t in_pstride, size_t in_bstride, int r, int npoly,
                  int nbatch, uint32_t* out, size_t out_pstride, size_t out_bstride, const EpiArgs& epi,
                  cudaStream_t st);

// Limb-domain kernels.
int launch_rescale(const fhe_ctx* ctx, const uint32_t* in, int logQ_in, uint32_t* out, int k, int npolys,
                   cudaStream_t st);
int launch_moddown(const fhe_ctx* ctx, const uint32_t* in, int logQ_in, uint32_t* out, int logQ_out, int npolys,
                   cudaStream_t st);
// b_polys > 0: b is that many polynomials reused for every group of b_polys outputs (broadcast)
int launch_addsub(const fhe_ctx* ctx, const uint32_t* a, const uint32_t* b, uint32_t* out, int logQ, int npolys,
                  int mode /*0 add,1 sub,2 neg(a)*/, cudaStream_t st, int b_polys = 0);
// out = in X^k (0 <= k < N), polys of ceil(logQ/32) limbs mod 2^logQ; out must not alias in.
int launch_monomial(const fhe_ctx* ctx, const uint32_t* in, uint32_t* out, int logQ, int k, int npolys,
                    cudaStream_t st);
int launch_mult_const(const fhe_ctx* ctx, const uint32_t* in, int32_t c, uint32_t* out, int logQ, int npolys,
                      cudaStream_t st);
int launch_add_const(const fhe_ctx* ctx, const uint32_t* in, uint32_t* out, int64_t value, const int64_t* values,
                     int shift, int logQ, int cnum, cudaStream_t st);
// out[l][n] = sign * in[l][i], kappa_g (X^i -> X^(i g)); polys of L limbs mod 2^logQ.
int launch_automorph(const fhe_ctx* ctx, const uint32_t* in, size_t in_pstride, uint32_t* out, size_t out_pstride,
                     int L, int logQ, uint32_t g, int npolys, cudaStream_t st);
int launch_automorph_small(const fhe_ctx* ctx, const int32_t* in, int32_t* out, uint32_t g, cudaStream_t st);
// keygen combine: out = (-t + e + (s_from << logP)) mod 2^bits, t two's complement limbs.
int launch_key_combine(const fhe_ctx* ctx, const uint32_t* t, int Lt, const int32_t* e, const uint32_t* sfrom,
                       int Ls, int logP, uint32_t* out, int bits, cudaStream_t st);

}  // namespace fhe
