// Negacyclic NTT / INTT per prime row (Sec. 2 Eq. negacyclic_ntt and
// Eq. negacyclic_intt; Sec. 5 "NTT-Based Polynomial Multiplication").
//
// The psi^j twist of Sec. 5 is merged into the twiddles: the forward transform
// is the Cooley-Tukey network with the bit-reversed table psi^brv(k) (natural
// input, bit-reversed output); the inverse is the Gentleman-Sande network with
// psi^-brv(k) (bit-reversed input, natural output) followed by the N^-1 scale.
// The bit-reversed order never leaves the device: pointwise products see both
// operands in the same order.
//
// Large rings use the two-pass decomposition of Sec. 5 ("Two-Pass NTT
// Decomposition", "Hierarchical Kernel Strategy"): the polynomial is viewed as
// an N1 x N2 matrix (N2 = 256 contiguous words per matrix row).  The first
// log N1 stages only pair elements in the same column, the last log N2 stages
// only pair elements in the same row, so each pass runs its stages on a tile
// held in shared memory.  The global twiddle step of the paper is absorbed:
// in the merged-twist CT network each stage already reads its own twiddle.
// Rings with N <= 8192 fit one CTA's shared memory and run in one pass.
#include "common.cuh"

namespace fhe {

constexpr int kRowLen = 256;   // N2
constexpr int kColTile = 32;   // columns per CTA in the column pass
constexpr int kRowTile = 4;    // matrix rows per CTA in the row pass

__device__ __forceinline__ void ct_bfly(uint32_t& x, uint32_t& y, uint32_t w, uint32_t wp, uint32_t q) {
  uint32_t v = shoup_mul(y, w, wp, q);
  uint32_t u = x;
  x = add_mod(u, v, q);
  y = sub_mod(u, v, q);
}
__device__ __forceinline__ void gs_bfly(uint32_t& x, uint32_t& y, uint32_t w, uint32_t wp, uint32_t q) {
  uint32_t u = x, v = y;
  x = add_mod(u, v, q);
  y = shoup_mul(u + q - v, w, wp, q);  // u - v + q < 2q < 2^32
}

// ---------------------------------------------------------------- one CTA
struct RowMap {
  int group_rows, group_stride;  // rows per group, group start stride (rows)
  __device__ __forceinline__ size_t row_of(int y) const {
    return (size_t)(y / group_rows) * group_stride + (y % group_rows);
  }
  __device__ __forceinline__ int prime_of(int y, int r) const { return (y % group_rows) % r; }
};

template <bool INV>
__global__ void __launch_bounds__(512) k_ntt_small(uint32_t* __restrict__ data, RowMap rm, int r, int logN,
                                                   const uint32_t* __restrict__ tw, const uint32_t* __restrict__ twp,
                                                   const uint32_t* __restrict__ qtab,
                                                   const uint32_t* __restrict__ nscale,
                                                   const uint32_t* __restrict__ nscale_sh) {
  extern __shared__ uint32_t s[];
  const int N = 1 << logN;
  const int p = rm.prime_of(blockIdx.x, r);
  const uint32_t q = __ldg(qtab + p);
  const uint32_t* w = tw + (size_t)p * N;
  const uint32_t* wp = twp + (size_t)p * N;
  uint32_t* a = data + rm.row_of(blockIdx.x) * N;
  for (int j = threadIdx.x; j < N; j += blockDim.x) s[j] = a[j];
  __syncthreads();
  const int half = N >> 1;
  if (!INV) {
    for (int m = 1, lt = logN - 1; m < N; m <<= 1, --lt) {
      for (int b = threadIdx.x; b < half; b += blockDim.x) {
        const int i = b >> lt;
        const int j = (i << (lt + 1)) + (b & ((1 << lt) - 1));
        ct_bfly(s[j], s[j + (1 << lt)], __ldg(w + m + i), __ldg(wp + m + i), q);
      }
      __syncthreads();
    }
    for (int j = threadIdx.x; j < N; j += blockDim.x) a[j] = s[j];
  } else {
    for (int h = half, lt = 0; h >= 1; h >>= 1, ++lt) {
      for (int b = threadIdx.x; b < half; b += blockDim.x) {
        const int i = b >> lt;
        const int j = (i << (lt + 1)) + (b & ((1 << lt) - 1));
        gs_bfly(s[j], s[j + (1 << lt)], __ldg(w + h + i), __ldg(wp + h + i), q);
      }
      __syncthreads();
    }
    const uint32_t sc = __ldg(nscale + p), scp = __ldg(nscale_sh + p);
    for (int j = threadIdx.x; j < N; j += blockDim.x) a[j] = shoup_mul(s[j], sc, scp, q);
  }
}

// ------------------------------------------------------------ column pass
// CTA: kColTile consecutive columns x0.. of one row (poly, prime), N1 x kColTile tile.
template <bool INV>
__global__ void __launch_bounds__(256) k_ntt_cols(uint32_t* __restrict__ data, RowMap rm, int r, int logN, int logN1,
                                                  const uint32_t* __restrict__ tw, const uint32_t* __restrict__ twp,
                                                  const uint32_t* __restrict__ qtab,
                                                  const uint32_t* __restrict__ nscale,
                                                  const uint32_t* __restrict__ nscale_sh) {
  extern __shared__ uint32_t s[];  // [N1][kColTile]
  const int N = 1 << logN, N1 = 1 << logN1;
  const int p = rm.prime_of(blockIdx.y, r);
  const uint32_t q = __ldg(qtab + p);
  const uint32_t* w = tw + (size_t)p * N;
  const uint32_t* wp = twp + (size_t)p * N;
  uint32_t* a = data + rm.row_of(blockIdx.y) * N + blockIdx.x * kColTile;
  for (int idx = threadIdx.x; idx < N1 * kColTile; idx += blockDim.x) {
    const int c = idx / kColTile, x = idx % kColTile;
    s[idx] = a[(size_t)c * kRowLen + x];
  }
  __syncthreads();
  const int nb = (N1 >> 1) * kColTile;
  if (!INV) {
    for (int m = 1, lt = logN1 - 1; m < N1; m <<= 1, --lt) {
      for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const int x = b % kColTile, bb = b / kColTile;
        const int i = bb >> lt;
        const int c = (i << (lt + 1)) + (bb & ((1 << lt) - 1));
        ct_bfly(s[c * kColTile + x], s[(c + (1 << lt)) * kColTile + x], __ldg(w + m + i), __ldg(wp + m + i), q);
      }
      __syncthreads();
    }
    for (int idx = threadIdx.x; idx < N1 * kColTile; idx += blockDim.x) {
      const int c = idx / kColTile, x = idx % kColTile;
      a[(size_t)c * kRowLen + x] = s[idx];
    }
  } else {
    for (int h = N1 >> 1, lt = 0; h >= 1; h >>= 1, ++lt) {
      for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const int x = b % kColTile, bb = b / kColTile;
        const int i = bb >> lt;
        const int c = (i << (lt + 1)) + (bb & ((1 << lt) - 1));
        gs_bfly(s[c * kColTile + x], s[(c + (1 << lt)) * kColTile + x], __ldg(w + h + i), __ldg(wp + h + i), q);
      }
      __syncthreads();
    }
    const uint32_t sc = __ldg(nscale + p), scp = __ldg(nscale_sh + p);
    for (int idx = threadIdx.x; idx < N1 * kColTile; idx += blockDim.x) {
      const int c = idx / kColTile, x = idx % kColTile;
      a[(size_t)c * kRowLen + x] = shoup_mul(s[idx], sc, scp, q);
    }
  }
}

// --------------------------------------------------------------- row pass
// CTA: kRowTile consecutive matrix rows c0.. of kRowLen contiguous words.
template <bool INV>
__global__ void __launch_bounds__(256) k_ntt_rows(uint32_t* __restrict__ data, RowMap rm, int r, int logN, int logN1,
                                                  const uint32_t* __restrict__ tw,
                                                  const uint32_t* __restrict__ twp,
                                                  const uint32_t* __restrict__ qtab) {
  __shared__ uint32_t s[kRowTile * kRowLen];
  const int N = 1 << logN, N1 = 1 << logN1;
  const int p = rm.prime_of(blockIdx.y, r);
  const uint32_t q = __ldg(qtab + p);
  const uint32_t* w = tw + (size_t)p * N;
  const uint32_t* wp = twp + (size_t)p * N;
  const int c0 = blockIdx.x * kRowTile;
  uint32_t* a = data + rm.row_of(blockIdx.y) * N + (size_t)c0 * kRowLen;
  for (int idx = threadIdx.x; idx < kRowTile * kRowLen; idx += blockDim.x) s[idx] = a[idx];
  __syncthreads();
  constexpr int kHalf = kRowLen / 2;
  constexpr int nb = kRowTile * kHalf;
  if (!INV) {
    // stages m = N1 .. N/2, t = kRowLen/2 .. 1
    for (int m = N1, lt = 7; lt >= 0; m <<= 1, --lt) {
      for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const int cr = b / kHalf, bj = b % kHalf;
        const int il = bj >> lt;
        const int jl = (il << (lt + 1)) + (bj & ((1 << lt) - 1));
        const int i = ((c0 + cr) << (7 - lt)) + il;  // global butterfly group
        ct_bfly(s[cr * kRowLen + jl], s[cr * kRowLen + jl + (1 << lt)], __ldg(w + m + i), __ldg(wp + m + i), q);
      }
      __syncthreads();
    }
  } else {
    // stages t = 1 .. kRowLen/2, h = N/2 .. N1
    for (int h = N >> 1, lt = 0; lt <= 7; h >>= 1, ++lt) {
      for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const int cr = b / kHalf, bj = b % kHalf;
        const int il = bj >> lt;
        const int jl = (il << (lt + 1)) + (bj & ((1 << lt) - 1));
        const int i = ((c0 + cr) << (7 - lt)) + il;
        gs_bfly(s[cr * kRowLen + jl], s[cr * kRowLen + jl + (1 << lt)], __ldg(w + h + i), __ldg(wp + h + i), q);
      }
      __syncthreads();
    }
  }
  for (int idx = threadIdx.x; idx < kRowTile * kRowLen; idx += blockDim.x) a[idx] = s[idx];
}

static int ntt_chunk(const fhe_ctx* ctx, uint32_t* data, RowMap rm, int rows, int r, bool inverse,
                     cudaStream_t st) {
  const int logN = ctx->prm.logN, N = ctx->N;
  const uint32_t* tw = inverse ? ctx->d_ipsi : ctx->d_psi;
  const uint32_t* twp = inverse ? ctx->d_ipsi_sh : ctx->d_psi_sh;
  ProfScope ps(ctx, inverse ? FHE_K_NTT_INV : FHE_K_NTT_FWD, logN <= 13 ? 1 : 2, st);
  if (logN <= 13) {
    const int threads = N / 2 < 32 ? 32 : (N / 2 > 512 ? 512 : N / 2);
    const size_t smem = (size_t)N * 4;
    if (inverse)
      k_ntt_small<true><<<rows, threads, smem, st>>>(data, rm, r, logN, tw, twp, ctx->d_q, ctx->d_nscale,
                                                      ctx->d_nscale_sh);
    else
      k_ntt_small<false><<<rows, threads, smem, st>>>(data, rm, r, logN, tw, twp, ctx->d_q, ctx->d_nscale,
                                                       ctx->d_nscale_sh);
    return FHE_OK;
  }
  const int logN1 = logN - 8, N1 = 1 << logN1;
  const size_t csmem = (size_t)N1 * kColTile * 4;
  dim3 gcols(kRowLen / kColTile, rows), grows(N1 / kRowTile, rows);
  if (!inverse) {
    k_ntt_cols<false><<<gcols, 256, csmem, st>>>(data, rm, r, logN, logN1, tw, twp, ctx->d_q, ctx->d_nscale,
                                                  ctx->d_nscale_sh);
    k_ntt_rows<false><<<grows, 256, 0, st>>>(data, rm, r, logN, logN1, tw, twp, ctx->d_q);
  } else {
    k_ntt_rows<true><<<grows, 256, 0, st>>>(data, rm, r, logN, logN1, tw, twp, ctx->d_q);
    k_ntt_cols<true><<<gcols, 256, csmem, st>>>(data, rm, r, logN, logN1, tw, twp, ctx->d_q, ctx->d_nscale,
                                                 ctx->d_nscale_sh);
  }
  return FHE_OK;
}

int launch_ntt(const fhe_ctx* ctx, uint32_t* data, int ngroups, int group_rows, int group_stride, int r,
               bool inverse, cudaStream_t st) {
  if (ngroups < 1 || group_rows < 1 || group_stride < group_rows || r < 1 || r > ctx->R) {
    set_error("ntt: bad row layout");
    return FHE_EINVAL;
  }
  // launch in chunks of whole groups so that grid.y stays <= 65535
  int per = 65535 / group_rows;
  if (per < 1) {
    set_error("ntt: %d rows per group exceed one launch", group_rows);
    return FHE_EINVAL;
  }
  const int N = ctx->N;
  for (int g0 = 0; g0 < ngroups; g0 += per) {
    const int ng = (ngroups - g0) < per ? (ngroups - g0) : per;
    RowMap rm{group_rows, group_stride};
    int rc = ntt_chunk(ctx, data + (size_t)g0 * group_stride * N, rm, ng * group_rows, r, inverse, st);
    if (rc) return rc;
  }
  return FHE_OK;
}

}  // namespace fhe
