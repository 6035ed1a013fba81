// The library's sampler for seeded key generation and encryption.
//
// The scheme draws a secret (uniform ternary or of a fixed Hamming weight),
// rounded Gaussian errors, uniform key parts and ternary ephemeral
// polynomials (Sec. 2 "Fully Homomorphic Encryption", Sec. 6 "Cryptographic
// Key Management"); the paper names no generator.  Every draw here comes from
// the counter-based generator Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
// "Parallel Random Numbers: As Easy as 1, 2, 3", SC 2011), so any word of
// any stream is computed independently of the others: on the host for key
// generation, in a kernel (one thread per four words) for the per-ciphertext
// randomness of encryption.
//
// Streams and rules (the same on host and device):
//   word j of stream (seed, tag0, tag1) = component j mod 4 of
//     Philox(counter (j/4 mod 2^32, j/2^34, tag0, tag1), key (seed lo, seed hi))
//   uniform mod 2^bits: limb l of coefficient n = word l N + n, top limb masked
//   ternary:            floor(3 w / 2^32) - 1
//   Hamming weight h:   partial Fisher-Yates shuffle, swap i <-> i + floor((N - i) w_i / 2^32)
//                       for i < h; the i-th chosen position is -1 if w_(h+i) is odd, else +1
//   rounded Gaussian:   thresholds T_k = floor(2^32 S_k / S_B), S_k the in-order double sums
//                       of exp(-k^2 / (2 sigma^2)) from k = -B, B = floor(6 sigma); the sample
//                       is the smallest k with w < T_k, or B
//   tags: 1 secret, 2/3 public key a/e, 4/5 relinearisation key a/e, 6/7 switching key a/e of
//         Galois element tag1, 8/9/10 encryption v/e0/e1 of ciphertext tag1
#include <math.h>

#include <vector>

#include "common.cuh"

namespace fhe {

// Ten Philox rounds on the counter c with key (k0, k1); c becomes the output block.
__host__ __device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = (uint32_t)p1;
    c[2] = n2;
    c[3] = (uint32_t)p0;
    k0 += 0x9E3779B9u;  // the key schedule's Weyl increments
    k1 += 0xBB67AE85u;
  }
}

__host__ __device__ __forceinline__ void stream_block(uint64_t seed, uint32_t tag0, uint32_t tag1, uint64_t blk,
                                                      uint32_t out[4]) {
  out[0] = (uint32_t)blk;
  out[1] = (uint32_t)(blk >> 32);
  out[2] = tag0;
  out[3] = tag1;
  philox4x32_10(out, (uint32_t)seed, (uint32_t)(seed >> 32));
}

__host__ __device__ __forceinline__ int8_t ternary_of(uint32_t w) {
  return (int8_t)((int)(((uint64_t)w * 3u) >> 32) - 1);
}

__host__ __device__ __forceinline__ int32_t gaussian_of(uint32_t w, const GaussTable& gt) {
  int lo = 0, hi = 2 * gt.B;  // first threshold above w
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (gt.thr[mid] <= w)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo - gt.B;
}

// ----------------------------------------------------------------- host side
int gauss_table(double sigma, GaussTable* gt) {
  if (!(sigma > 0.0) || sigma > kMaxGaussSigma) return FHE_EINVAL;
  const int B = (int)floor(6.0 * sigma);
  if (B < 1 || B > kMaxGaussB) return FHE_EINVAL;
  std::vector<double> run(2 * B + 1);
  double acc = 0.0;
  for (int k = -B; k <= B; ++k) {
    acc += exp(-(double)(k * k) / (2.0 * sigma * sigma));
    run[k + B] = acc;
  }
  const double total = run[2 * B];
  for (int i = 0; i < 2 * B; ++i) gt->thr[i] = (uint32_t)floor(run[i] / total * 4294967296.0);
  gt->B = B;
  return FHE_OK;
}

void sample_words(uint64_t seed, uint32_t tag0, uint32_t tag1, size_t count, uint32_t* out) {
  uint32_t blk[4];
  for (size_t j = 0; j < count; ++j) {
    if ((j & 3) == 0) stream_block(seed, tag0, tag1, j >> 2, blk);
    out[j] = blk[j & 3];
  }
}

void sample_uniform_limbs(uint64_t seed, uint32_t tag0, uint32_t tag1, int n, int bits, uint32_t* out) {
  const int L = limbs_for_bits(bits);
  sample_words(seed, tag0, tag1, (size_t)L * n, out);
  const int top = bits - 32 * (L - 1);
  if (top < 32)
    for (int i = 0; i < n; ++i) out[(size_t)(L - 1) * n + i] &= (1u << top) - 1u;
}

void sample_ternary(uint64_t seed, uint32_t tag0, uint32_t tag1, int n, int8_t* out) {
  std::vector<uint32_t> w(n);
  sample_words(seed, tag0, tag1, n, w.data());
  for (int i = 0; i < n; ++i) out[i] = ternary_of(w[i]);
}

void sample_sparse_ternary(uint64_t seed, uint32_t tag0, uint32_t tag1, int n, int h, int8_t* out) {
  std::vector<uint32_t> w(2 * (size_t)h);
  sample_words(seed, tag0, tag1, w.size(), w.data());
  std::vector<int> perm(n);
  for (int i = 0; i < n; ++i) perm[i] = i, out[i] = 0;
  for (int i = 0; i < h; ++i) {
    const int r = i + (int)(((uint64_t)(n - i) * w[i]) >> 32);
    const int t = perm[i];
    perm[i] = perm[r];
    perm[r] = t;
    out[perm[i]] = (w[h + i] & 1u) ? -1 : 1;
  }
}

void sample_gaussian(uint64_t seed, uint32_t tag0, uint32_t tag1, int n, const GaussTable& gt, int32_t* out) {
  std::vector<uint32_t> w(n);
  sample_words(seed, tag0, tag1, n, w.data());
  for (int i = 0; i < n; ++i) out[i] = gaussian_of(w[i], gt);
}

// --------------------------------------------------------------- device side
// Encryption randomness of cnum ciphertexts: v (ternary, tag 8), e0, e1
// (Gaussian, tags 9 and 10), tag1 = the ciphertext's index.  One thread per
// Philox block, i.e. four consecutive coefficients; grid (blocks, cnum, 3).
__global__ void k_sample_enc(uint64_t seed, int N, int8_t* __restrict__ v, int32_t* __restrict__ e0,
                             int32_t* __restrict__ e1, GaussTable gt) {
  const int blk = blockIdx.x * blockDim.x + threadIdx.x;
  if (4 * blk >= N) return;
  const int c = blockIdx.y, which = blockIdx.z;
  uint32_t w[4];
  stream_block(seed, kTagEncV + which, (uint32_t)c, (uint64_t)blk, w);
  const size_t o = (size_t)c * N + 4 * (size_t)blk;
  if (which == 0) {
    char4 t;
    t.x = ternary_of(w[0]);
    t.y = ternary_of(w[1]);
    t.z = ternary_of(w[2]);
    t.w = ternary_of(w[3]);
    *reinterpret_cast<char4*>(v + o) = t;
  } else {
    int4 t = make_int4(gaussian_of(w[0], gt), gaussian_of(w[1], gt), gaussian_of(w[2], gt), gaussian_of(w[3], gt));
    *reinterpret_cast<int4*>((which == 1 ? e0 : e1) + o) = t;
  }
}

int launch_sample_enc(const fhe_ctx* ctx, uint64_t seed, int cnum, int8_t* v, int32_t* e0, int32_t* e1,
                      cudaStream_t st) {
  const int N = ctx->N, threads = 128;
  const int blocks = (N / 4 + threads - 1) / threads;
  ProfScope ps(ctx, FHE_K_LIMB, 1, st);
  k_sample_enc<<<dim3(blocks, cnum, 3), threads, 0, st>>>(seed, N, v, e0, e1, ctx->gauss);
  return FHE_OK;
}

}  // namespace fhe

extern "C" {

int fhe_sample(uint64_t seed, uint32_t tag0, uint32_t tag1, int kind, int n, int param, double sigma, void* out) {
  using namespace fhe;
  if (!out || n < 1 || n > (1 << 24)) {
    set_error("sample: null output or n out of range");
    return FHE_EINVAL;
  }
  switch (kind) {
    case FHE_SAMPLE_UNIFORM:
      if (param < 1 || param > 32 * kMaxLimbs) break;
      sample_uniform_limbs(seed, tag0, tag1, n, param, (uint32_t*)out);
      return FHE_OK;
    case FHE_SAMPLE_TERNARY:
      sample_ternary(seed, tag0, tag1, n, (int8_t*)out);
      return FHE_OK;
    case FHE_SAMPLE_HWT:
      if (param < 1 || param > n) break;
      sample_sparse_ternary(seed, tag0, tag1, n, param, (int8_t*)out);
      return FHE_OK;
    case FHE_SAMPLE_GAUSSIAN: {
      GaussTable gt;
      if (gauss_table(sigma, &gt) != FHE_OK) break;
      sample_gaussian(seed, tag0, tag1, n, gt, (int32_t*)out);
      return FHE_OK;
    }
    default:
      break;
  }
  set_error("sample: bad kind %d or parameter %d (sigma %g)", kind, param, sigma);
  return FHE_EINVAL;
}

}  // extern "C"
