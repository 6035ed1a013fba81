// Plaintext encoding on the GPU.
//
// CKKS (Sec. 2 "Fast Fourier Transform"; HEAAN slots as adopted in Sec. 6):
// slot j of an integer plaintext m(X) is m(zeta^(5^j mod 2N)) / Delta with
// zeta = exp(i pi / N), j < N/2 (full packing).  Writing a_i = m_i zeta^i, the
// values at all odd powers are a DFT: m(zeta^(2k+1)) = sum_i a_i omega^(ik),
// omega = zeta^2.  Encoding places Delta z_j at index (5^j - 1)/2 and its
// conjugate at (2N - 5^j - 1)/2 (the conjugate root), runs the inverse DFT,
// untwists by zeta^(-i), divides by N and rounds the real part to the nearest
// integer (ties to even), written as logQ-bit two's-complement limbs.
// Decoding converts centred limbs to double, twists, runs the forward DFT and
// gathers the rotation-group order.  The DFTs are radix-2 Stockham passes in
// double precision (one launch per stage, self-sorting, ping-pong buffers).
//
// BGV slot batching (Sec. 2 "Chinese Remainder Theorem", the polynomial CRT):
// for a prime t = 1 (mod 2N), X^N + 1 = prod_k (X - psi^(2k+1)) mod t with psi
// a primitive 2N-th root of unity, and m -> (m(psi^(2k+1)))_k is a ring
// isomorphism onto Z_t^N, so slot-wise products are ciphertext products.
// psi = g^((t-1)/(2N)) with g the smallest primitive root mod t.  One CTA per
// polynomial runs the cyclic NTT of the twisted coefficients in shared memory
// (bit-reversed load, in-place decimation-in-time stages).
#include <math.h>

#include <vector>

#include "common.cuh"

namespace fhe {

__device__ __forceinline__ uint32_t pow5_mod(uint32_t j, uint32_t two_n) {
  uint32_t r = 1, b = 5 % two_n;
  while (j) {
    if (j & 1u) r = (uint32_t)(((uint64_t)r * b) & (two_n - 1));
    b = (uint32_t)(((uint64_t)b * b) & (two_n - 1));
    j >>= 1;
  }
  return r;
}

// One radix-2 Stockham stage over every polynomial of the batch: l = N / 2^(s+1), m = 2^s.
__global__ void k_fft_stage(const double2* __restrict__ x, double2* __restrict__ y, int logN, int l, int m,
                            double sign, int cnum) {
  const int N = 1 << logN, half = N >> 1;
  const size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (size_t)cnum * half) return;
  const int b = (int)(id / half), t = (int)(id - (size_t)b * half);
  const int j = t / m, k = t - j * m;
  const double2* xb = x + (size_t)b * N;
  double2* yb = y + (size_t)b * N;
  const double2 c0 = xb[k + j * m], c1 = xb[k + j * m + l * m];
  double s, c;
  sincospi((double)j / (double)l, &s, &c);
  s *= sign;
  const double dx = c0.x - c1.x, dy = c0.y - c1.y;
  yb[k + 2 * j * m] = make_double2(c0.x + c1.x, c0.y + c1.y);
  yb[k + 2 * j * m + m] = make_double2(c * dx - s * dy, c * dy + s * dx);
}

// vals[(e - 1)/2] = Delta z_j, vals[(2N - e - 1)/2] = Delta conj(z_j), e = 5^j mod 2N.
__global__ void k_ckks_scatter(const double2* __restrict__ z, double2* __restrict__ vals, int logN, double delta,
                               int cnum) {
  const int N = 1 << logN, n = N >> 1;
  const size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (size_t)cnum * n) return;
  const int b = (int)(id / n), j = (int)(id - (size_t)b * n);
  const uint32_t e = pow5_mod((uint32_t)j, 2u * N);
  const double2 v = z[id];
  vals[(size_t)b * N + (e - 1) / 2] = make_double2(delta * v.x, delta * v.y);
  vals[(size_t)b * N + (2u * N - e - 1) / 2] = make_double2(delta * v.x, -delta * v.y);
}

// m_i = rint(Re(Y_i zeta^(-i)) / N) as two's-complement limbs mod 2^logQ (|m_i| <= Delta max|z| < 2^62).
__global__ void k_ckks_encode_finish(const double2* __restrict__ Y, uint32_t* __restrict__ pt, int logN, int L,
                                     int logQ, int cnum) {
  const int N = 1 << logN;
  const size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (size_t)cnum * N) return;
  const int b = (int)(id / N), i = (int)(id - (size_t)b * N);
  double s, c;
  sincospi((double)i / (double)N, &s, &c);
  const double2 v = Y[id];
  const long long m = llrint((v.x * c + v.y * s) / (double)N);
  const uint32_t ext = m < 0 ? 0xFFFFFFFFu : 0u;
  uint32_t* o = pt + (size_t)b * L * N + i;
  for (int l = 0; l < L; ++l) {
    uint32_t w = l == 0 ? (uint32_t)m : (l == 1 ? (uint32_t)((unsigned long long)m >> 32) : ext);
    const int rem = logQ - 32 * l;
    if (rem < 32) w &= rem <= 0 ? 0u : ((1u << rem) - 1u);
    o[(size_t)l * N] = w;
  }
}

// a_i = m_i zeta^i, m_i the signed value of L-limb two's complement (as decryption writes it).
// h = the highest limb that differs from the sign extension; the window of limbs h, h-1, h-2 with
// the extension above carries the value to double precision: T = w_h - 2^32 [negative] is exact,
// then (T 2^32 + w_(h-1)) 2^32 + w_(h-2), scaled by 2^(32 (h-2)).
__global__ void k_ckks_decode_load(const uint32_t* __restrict__ pt, double2* __restrict__ a, int logN, int L,
                                   int cnum) {
  const int N = 1 << logN;
  const size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (size_t)cnum * N) return;
  const int b = (int)(id / N), i = (int)(id - (size_t)b * N);
  const uint32_t* x = pt + (size_t)b * L * N + i;
  const bool neg = (x[(size_t)(L - 1) * N] >> 31) != 0;
  const uint32_t ext = neg ? 0xFFFFFFFFu : 0u;
  int h = L - 1;
  while (h >= 0 && x[(size_t)h * N] == ext) --h;
  double m;
  if (h < 0) {
    m = neg ? -1.0 : 0.0;
  } else {
    const double t = (double)((long long)x[(size_t)h * N] - (neg ? 4294967296LL : 0LL));
    const double w1 = h >= 1 ? (double)x[(size_t)(h - 1) * N] : 0.0;
    const double w2 = h >= 2 ? (double)x[(size_t)(h - 2) * N] : 0.0;
    m = ldexp((t * 4294967296.0 + w1) * 4294967296.0 + w2, 32 * (h - 2));
  }
  double s, c;
  sincospi((double)i / (double)N, &s, &c);
  a[id] = make_double2(m * c, m * s);
}

// z_j = vals[(5^j - 1)/2] / Delta
__global__ void k_ckks_gather(const double2* __restrict__ vals, double2* __restrict__ z, int logN, double inv_delta,
                              int cnum) {
  const int N = 1 << logN, n = N >> 1;
  const size_t id = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (size_t)cnum * n) return;
  const int b = (int)(id / n), j = (int)(id - (size_t)b * n);
  const uint32_t e = pow5_mod((uint32_t)j, 2u * N);
  const double2 v = vals[(size_t)b * N + (e - 1) / 2];
  z[id] = make_double2(v.x * inv_delta, v.y * inv_delta);
}

// Stockham DFT of cnum length-N rows: sign -1 forward (e^(-2 pi i jk/N)), +1 inverse (unscaled).
// x is the input and is overwritten; the result is in *res (x or y).
static void fft(const fhe_ctx* ctx, double2* x, double2* y, int cnum, double sign, double2** res, cudaStream_t st) {
  const int logN = ctx->prm.logN, N = ctx->N;
  const size_t work = (size_t)cnum * (N / 2);
  const int threads = 256;
  const unsigned blocks = (unsigned)((work + threads - 1) / threads);
  for (int l = N / 2, m = 1; l >= 1; l >>= 1, m <<= 1) {
    k_fft_stage<<<blocks, threads, 0, st>>>(x, y, logN, l, m, sign, cnum);
    double2* t = x;
    x = y;
    y = t;
  }
  *res = x;
}

// ------------------------------------------------------------- BGV slots
// Cyclic NTT mod t of length N in shared memory on one polynomial per CTA:
//   forward: out[k] = sum_i (in[i] psi^i) omega^(ik) = m(psi^(2k+1))          (decode)
//   inverse: out[i] = N^-1 psi^(-i) sum_k in[k] omega^(-ik)                    (encode)
// tab: [0, N) psi^i, [N, 2N) N^-1 psi^(-i), [2N, 2N + N/2) omega^i, [2N + N/2, 3N) omega^(-i).
__global__ void __launch_bounds__(1024) k_bgv_slots(const uint32_t* __restrict__ in, size_t in_stride,
                                                    uint32_t* __restrict__ out, size_t out_stride, int logN,
                                                    uint32_t t, const uint32_t* __restrict__ tab, int inverse) {
  extern __shared__ uint32_t sv[];
  const int N = 1 << logN;
  const uint32_t* src = in + (size_t)blockIdx.x * in_stride;
  uint32_t* dst = out + (size_t)blockIdx.x * out_stride;
  const uint32_t* w = tab + 2 * N + (inverse ? N / 2 : 0);
  // bit-reversed load (decimation in time); the forward transform twists first
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    uint32_t v = src[i] % t;
    if (!inverse) v = (uint32_t)(((uint64_t)v * __ldg(tab + i)) % t);
    sv[__brev((uint32_t)i) >> (32 - logN)] = v;
  }
  __syncthreads();
  for (int len = 2; len <= N; len <<= 1) {
    const int hl = len >> 1, step = N / len;
    for (int q = threadIdx.x; q < N / 2; q += blockDim.x) {
      const int blk = q / hl, j = q - blk * hl;
      const int p0 = blk * len + j, p1 = p0 + hl;
      const uint32_t u = sv[p0];
      const uint32_t v = (uint32_t)(((uint64_t)sv[p1] * __ldg(w + j * step)) % t);
      sv[p0] = u + v >= t ? u + v - t : u + v;
      sv[p1] = u >= v ? u - v : u + t - v;
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    uint32_t v = sv[i];
    if (inverse) v = (uint32_t)(((uint64_t)v * __ldg(tab + N + i)) % t);
    dst[i] = v;
  }
}

static uint32_t powmod32(uint64_t b, uint64_t e, uint64_t m) {
  uint64_t r = 1 % m;
  b %= m;
  while (e) {
    if (e & 1) r = r * b % m;
    b = b * b % m;
    e >>= 1;
  }
  return (uint32_t)r;
}

static bool is_prime32(uint32_t n) {
  if (n < 2) return false;
  for (uint32_t d = 2; (uint64_t)d * d <= n; ++d)
    if (n % d == 0) return false;
  return true;
}

// The slot tables of the context's t (BGV, prime t = 1 mod 2N), built on first use.
static int bgv_slot_tables(fhe_ctx* ctx) {
  if (ctx->d_bgv_slots) return FHE_OK;
  const uint32_t t = ctx->prm.t;
  const uint64_t N = (uint64_t)ctx->N;
  if (ctx->prm.scheme != FHE_SCHEME_BGV || !is_prime32(t) || (t - 1) % (2 * N) != 0 || ctx->prm.logN > 15) {
    set_error("bgv slots: need a BGV context with a prime t = 1 mod 2N and N <= 2^15 (t = %u, N = %llu)", t,
              (unsigned long long)N);
    return FHE_EINVAL;
  }
  // smallest primitive root g: g^((t-1)/p) != 1 for every prime p | t - 1
  std::vector<uint32_t> pf;
  uint32_t r = t - 1;
  for (uint32_t d = 2; (uint64_t)d * d <= r; ++d)
    if (r % d == 0) {
      pf.push_back(d);
      while (r % d == 0) r /= d;
    }
  if (r > 1) pf.push_back(r);
  uint32_t g = 2;
  for (;; ++g) {
    bool ok = true;
    for (uint32_t p : pf)
      if (powmod32(g, (t - 1) / p, t) == 1) ok = false;
    if (ok) break;
  }
  const uint32_t psi = powmod32(g, (t - 1) / (2 * N), t), psi_inv = powmod32(psi, t - 2, t);
  const uint32_t n_inv = powmod32((uint32_t)(N % t), t - 2, t);
  const uint32_t om = (uint32_t)((uint64_t)psi * psi % t), om_inv = (uint32_t)((uint64_t)psi_inv * psi_inv % t);
  std::vector<uint32_t> tab(3 * N);
  uint64_t a = 1, ai = n_inv, o = 1, oi = 1;
  for (uint64_t i = 0; i < N; ++i) {
    tab[i] = (uint32_t)a;
    tab[N + i] = (uint32_t)ai;
    a = a * psi % t;
    ai = ai * psi_inv % t;
  }
  for (uint64_t i = 0; i < N / 2; ++i) {
    tab[2 * N + i] = (uint32_t)o;
    tab[2 * N + N / 2 + i] = (uint32_t)oi;
    o = o * om % t;
    oi = oi * om_inv % t;
  }
  uint32_t* d = (uint32_t*)ctx_alloc(ctx, tab.size() * 4);
  if (!d) {
    set_error("bgv slots: table allocation failed");
    return FHE_ENOMEM;
  }
  if (cudaMemcpy(d, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
    set_error("bgv slots: table upload failed");
    return FHE_ECUDA;
  }
  ctx->d_bgv_slots = d;
  cudaFuncSetAttribute(k_bgv_slots, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(N * 4));
  return FHE_OK;
}

}  // namespace fhe

using namespace fhe;

extern "C" {

int fhe_ckks_encode(fhe_ctx* ctx, const double* z, int cnum, int log_scale, int logQ, uint32_t* pt, void* ws,
                    size_t ws_bytes, void* stream) {
  if (!ctx || !z || !pt || cnum < 1 || ctx->prm.scheme != FHE_SCHEME_CKKS || logQ < 1 || logQ > ctx->prm.logQ ||
      log_scale < 0 || log_scale > 62 || ctx->prm.logN < 2) {
    set_error("ckks_encode: bad arguments (CKKS, 1 <= logQ <= top, 0 <= log_scale <= 62)");
    return FHE_EINVAL;
  }
  const int N = ctx->N;
  const size_t need = 2 * (size_t)cnum * N * sizeof(double2);
  if (!ws || ws_bytes < need || ((uintptr_t)ws & 255)) {
    set_error("ckks_encode: workspace of %zu bytes too small or misaligned (need %zu)", ws_bytes, need);
    return FHE_EWORKSPACE;
  }
  cudaStream_t st = (cudaStream_t)stream;
  double2* x = (double2*)ws;
  double2* y = x + (size_t)cnum * N;
  ProfScope ps(ctx, FHE_K_LIMB, 2 + ctx->prm.logN, st);
  const int threads = 256;
  const size_t nh = (size_t)cnum * (N / 2), nf = (size_t)cnum * N;
  k_ckks_scatter<<<(unsigned)((nh + threads - 1) / threads), threads, 0, st>>>((const double2*)z, x, ctx->prm.logN,
                                                                               ldexp(1.0, log_scale), cnum);
  double2* res = nullptr;
  fft(ctx, x, y, cnum, -1.0, &res, st);
  k_ckks_encode_finish<<<(unsigned)((nf + threads - 1) / threads), threads, 0, st>>>(
      res, pt, ctx->prm.logN, limbs_for_bits(logQ), logQ, cnum);
  FHE_CHECK_CUDA(cudaGetLastError());
  return FHE_OK;
}

int fhe_ckks_decode(fhe_ctx* ctx, const uint32_t* pt, int cnum, int logQ, double log_scale, double* z, void* ws,
                    size_t ws_bytes, void* stream) {
  if (!ctx || !z || !pt || cnum < 1 || ctx->prm.scheme != FHE_SCHEME_CKKS || logQ < 1 || logQ > ctx->prm.logQ ||
      !(log_scale >= 0.0 && log_scale < 1000.0)) {
    set_error("ckks_decode: bad arguments");
    return FHE_EINVAL;
  }
  const int N = ctx->N;
  const size_t need = 2 * (size_t)cnum * N * sizeof(double2);
  if (!ws || ws_bytes < need || ((uintptr_t)ws & 255)) {
    set_error("ckks_decode: workspace of %zu bytes too small or misaligned (need %zu)", ws_bytes, need);
    return FHE_EWORKSPACE;
  }
  cudaStream_t st = (cudaStream_t)stream;
  double2* x = (double2*)ws;
  double2* y = x + (size_t)cnum * N;
  ProfScope ps(ctx, FHE_K_LIMB, 2 + ctx->prm.logN, st);
  const int threads = 256;
  const size_t nh = (size_t)cnum * (N / 2), nf = (size_t)cnum * N;
  k_ckks_decode_load<<<(unsigned)((nf + threads - 1) / threads), threads, 0, st>>>(pt, x, ctx->prm.logN,
                                                                                  limbs_for_bits(logQ), cnum);
  double2* res = nullptr;
  fft(ctx, x, y, cnum, +1.0, &res, st);
  k_ckks_gather<<<(unsigned)((nh + threads - 1) / threads), threads, 0, st>>>(res, (double2*)z, ctx->prm.logN,
                                                                              exp2(-log_scale), cnum);
  FHE_CHECK_CUDA(cudaGetLastError());
  return FHE_OK;
}

int fhe_bgv_encode(fhe_ctx* ctx, const uint32_t* slots, int cnum, uint32_t* pt, size_t pt_stride, void* stream) {
  if (!ctx || !slots || !pt || cnum < 1 || cnum > 65535 || pt_stride < (size_t)(ctx ? ctx->N : 0)) {
    set_error("bgv_encode: bad arguments");
    return FHE_EINVAL;
  }
  int rc = bgv_slot_tables(ctx);
  if (rc != FHE_OK) return rc;
  const int N = ctx->N;
  ProfScope ps(ctx, FHE_K_LIMB, 1, (cudaStream_t)stream);
  k_bgv_slots<<<cnum, N / 2 < 1024 ? N / 2 : 1024, (size_t)N * 4, (cudaStream_t)stream>>>(
      slots, (size_t)N, pt, pt_stride, ctx->prm.logN, ctx->prm.t, ctx->d_bgv_slots, 1);
  FHE_CHECK_CUDA(cudaGetLastError());
  return FHE_OK;
}

int fhe_bgv_decode(fhe_ctx* ctx, const uint32_t* pt, size_t pt_stride, int cnum, uint32_t* slots, void* stream) {
  if (!ctx || !slots || !pt || cnum < 1 || cnum > 65535 || pt_stride < (size_t)(ctx ? ctx->N : 0)) {
    set_error("bgv_decode: bad arguments");
    return FHE_EINVAL;
  }
  int rc = bgv_slot_tables(ctx);
  if (rc != FHE_OK) return rc;
  const int N = ctx->N;
  ProfScope ps(ctx, FHE_K_LIMB, 1, (cudaStream_t)stream);
  k_bgv_slots<<<cnum, N / 2 < 1024 ? N / 2 : 1024, (size_t)N * 4, (cudaStream_t)stream>>>(
      pt, pt_stride, slots, (size_t)N, ctx->prm.logN, ctx->prm.t, ctx->d_bgv_slots, 0);
  FHE_CHECK_CUDA(cudaGetLastError());
  return FHE_OK;
}

}  // extern "C"
