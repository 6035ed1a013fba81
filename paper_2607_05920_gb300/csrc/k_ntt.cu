// Negacyclic NTT / INTT per prime row (Sec. 2 Eq. negacyclic_ntt and
// Eq. negacyclic_intt; Sec. 5 "NTT-Based Polynomial Multiplication").
//
// The psi^j twist of Sec. 5 is merged into the twiddles: the forward transform
// is the Cooley-Tukey network with the bit-reversed table psi^brv(k) (natural
// input, bit-reversed output); the inverse is the Gentleman-Sande network with
// psi^-brv(k) (bit-reversed input, natural output).  The inverse leaves out the
// N^-1 scale (and the 2^32 that undoes the Montgomery products' 2^-32) and its
// final reduction: every inverse transform feeds a reconstruction whose first
// step multiplies each residue by a per-prime constant, which absorbs both.
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
// Rings with N <= 4096 run in one CTA (all stages in shared memory).
//
// Above that, a ring product (Sec. 5 pipeline: forward NTTs, pointwise
// products, inverse NTTs) is three launches: the forward column stages, one
// fused pass that finishes the forward transforms in each 256-word row, forms
// the products there and runs the inverse row stages (the transform-domain
// values never reach global memory), and the inverse column stages.  Each
// of these kernels is a job function plus a one-group launch; the work-table
// kernels at the end run the same jobs for many groups of ring products (any
// ring sizes from 2^13 to 2^16 and prime counts) in one launch each.
#include "common.cuh"

namespace fhe {

constexpr int kRowLen = 256;   // N2

// Lazy butterflies (Harvey, "Faster arithmetic for number-theoretic
// transforms", 2014): with q < 2^30, 4q fits a word, so values travel between
// stages only partly reduced and each butterfly does one conditional
// subtraction.  Forward (CT): x, y in [0, 4q) -> [0, 4q).  Inverse (GS):
// x, y in [0, 2q) -> [0, 2q).  Shoup products with a lazy result in [0, 2q).
__device__ __forceinline__ void ct_bfly(uint32_t& x, uint32_t& y, uint32_t w, uint32_t wp, uint32_t q) {
  const uint32_t q2 = 2u * q;
  const uint32_t u = min(x, x - q2);                // [0, 2q): x - 2q wraps above x when x < 2q
  const uint32_t t = shoup_mul_lazy(y, w, wp, q);   // [0, 2q)
  x = u + t;                                        // [0, 4q)
  y = u - t + q2;                                   // (0, 4q)
}
__device__ __forceinline__ void gs_bfly(uint32_t& x, uint32_t& y, uint32_t w, uint32_t wp, uint32_t q) {
  const uint32_t q2 = 2u * q;
  const uint32_t s = x + y;                         // [0, 4q)
  const uint32_t d = x - y + q2;                    // (0, 4q)
  x = min(s, s - q2);                               // [0, 2q)
  y = shoup_mul_lazy(d, w, wp, q);                  // [0, 2q)
}
// [0, 4q) -> [0, q)
__device__ __forceinline__ uint32_t reduce4(uint32_t x, uint32_t q) {
  x = min(x, x - 2u * q);
  return min(x, x - q);
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
                                                   const uint2* __restrict__ tw,
                                                   const uint32_t* __restrict__ qtab) {
  extern __shared__ uint32_t s[];
  const int N = 1 << logN;
  const int p = rm.prime_of(blockIdx.x, r);
  const uint32_t q = __ldg(qtab + p);
  const uint2* w = tw + (size_t)p * N;
  uint32_t* a = data + rm.row_of(blockIdx.x) * N;
  for (int j = threadIdx.x; j < N; j += blockDim.x) s[j] = a[j];
  __syncthreads();
  const int half = N >> 1;
  if (!INV) {
    for (int m = 1, lt = logN - 1; m < N; m <<= 1, --lt) {
      for (int b = threadIdx.x; b < half; b += blockDim.x) {
        const int i = b >> lt;
        const int j = (i << (lt + 1)) + (b & ((1 << lt) - 1));
        const uint2 t2 = __ldg(w + m + i);
        ct_bfly(s[j], s[j + (1 << lt)], t2.x, t2.y, q);
      }
      __syncthreads();
    }
    for (int j = threadIdx.x; j < N; j += blockDim.x) a[j] = reduce4(s[j], q);
  } else {
    for (int h = half, lt = 0; h >= 1; h >>= 1, ++lt) {
      for (int b = threadIdx.x; b < half; b += blockDim.x) {
        const int i = b >> lt;
        const int j = (i << (lt + 1)) + (b & ((1 << lt) - 1));
        const uint2 t2 = __ldg(w + h + i);
        gs_bfly(s[j], s[j + (1 << lt)], t2.x, t2.y, q);
      }
      __syncthreads();
    }
    // left in [0, 2q) and unscaled: the reconstruction folds N^-1 2^32 into its first product
    for (int j = threadIdx.x; j < N; j += blockDim.x) a[j] = s[j];
  }
}

// ------------------------------------------------------------ column pass
// The first log N1 stages of the forward transform (last of the inverse) pair
// elements in the same column of the N1 x 256 matrix.  A CTA takes 32
// adjacent columns; each column is split over N1/16 threads that keep 16
// elements in registers.  Layout A: thread j0 holds rows j0 + (N1/16) k
// (k < 16), so four stages (row distances N1/2 .. N1/16) run in registers;
// layout B after one shared-memory exchange: rows 16 j0 + j (j < 16) for
// the remaining stages (distances N1/32 .. 1).  A warp always spans 32
// columns of one row: global accesses are 128-byte coalesced, shared-memory
// accesses conflict-free, and the twiddle of a butterfly depends only on the
// row, so twiddle loads are warp-wide broadcasts.
// One column job: the first log N1 forward stages of the 32 columns [32 bx, 32 bx + 32) of row y
// of the row map (N = N1 x 256 words), run by 2 N1 threads (tid < 2 N1) over the N1 x 32 words of
// shared memory at s.  Contains one barrier of the whole CTA, so every thread of the CTA calls it.
template <int LOGN1>
__device__ __forceinline__ void cols_fwd_job(uint32_t* __restrict__ data, RowMap rm, int r, int N, int bx, int y,
                                             int tid, uint32_t* s, const uint2* __restrict__ tw,
                                             const uint32_t* __restrict__ qtab) {
  constexpr int N1 = 1 << LOGN1, TPC = N1 / 16;
  const int col = tid & 31, j0 = tid >> 5;
  const int p = rm.prime_of(y, r);
  const uint32_t q = __ldg(qtab + p);
  const uint2* w = tw + (size_t)p * N;
  uint32_t* a = data + rm.row_of(y) * N + bx * 32 + col;
  uint32_t x[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) x[k] = a[(size_t)(j0 + TPC * k) * kRowLen];
  // layout A: distance TPC*h rows, stage index m = 8/h, group k/(2h)
#pragma unroll
  for (int h = 8, m = 1; h >= 1; h >>= 1, m <<= 1) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      if (k & h) continue;
      const int i = k / (2 * h);
      const uint2 t2 = __ldg(w + m + i);
      ct_bfly(x[k], x[k + h], t2.x, t2.y, q);
    }
  }
#pragma unroll
  for (int k = 0; k < 16; ++k) s[(j0 + TPC * k) * 32 + col] = x[k];
  __syncthreads();
#pragma unroll
  for (int j = 0; j < 16; ++j) x[j] = s[(16 * j0 + j) * 32 + col];
  // layout B: distance h rows (h = N1/32 .. 1), stage index N1/(2h), group (16 j0 + j)/(2h)
#pragma unroll
  for (int h = N1 / 32; h >= 1; h >>= 1) {
    const int m = N1 / (2 * h);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if (j & h) continue;
      const int i = j0 * (8 / h) + j / (2 * h);
      const uint2 t2 = __ldg(w + m + i);
      ct_bfly(x[j], x[j + h], t2.x, t2.y, q);
    }
  }
#pragma unroll
  for (int j = 0; j < 16; ++j) a[(size_t)(16 * j0 + j) * kRowLen] = x[j];
}

// The inverse column job (the last log N1 inverse stages), arguments as cols_fwd_job.
template <int LOGN1>
__device__ __forceinline__ void cols_inv_job(uint32_t* __restrict__ data, RowMap rm, int r, int N, int bx, int y,
                                             int tid, uint32_t* s, const uint2* __restrict__ tw,
                                             const uint32_t* __restrict__ qtab) {
  constexpr int N1 = 1 << LOGN1, TPC = N1 / 16;
  const int col = tid & 31, j0 = tid >> 5;
  const int p = rm.prime_of(y, r);
  const uint32_t q = __ldg(qtab + p);
  const uint2* w = tw + (size_t)p * N;
  uint32_t* a = data + rm.row_of(y) * N + bx * 32 + col;
  uint32_t x[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) x[j] = a[(size_t)(16 * j0 + j) * kRowLen];
#pragma unroll
  for (int h = 1; h <= N1 / 32; h <<= 1) {
    const int m = N1 / (2 * h);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if (j & h) continue;
      const int i = j0 * (8 / h) + j / (2 * h);
      const uint2 t2 = __ldg(w + m + i);
      gs_bfly(x[j], x[j + h], t2.x, t2.y, q);
    }
  }
#pragma unroll
  for (int j = 0; j < 16; ++j) s[(16 * j0 + j) * 32 + col] = x[j];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 16; ++k) x[k] = s[(j0 + TPC * k) * 32 + col];
#pragma unroll
  for (int h = 1, m = 8; h <= 8; h <<= 1, m >>= 1) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      if (k & h) continue;
      const int i = k / (2 * h);
      const uint2 t2 = __ldg(w + m + i);
      gs_bfly(x[k], x[k + h], t2.x, t2.y, q);
    }
  }
  // left in [0, 2q) and unscaled: the reconstruction folds N^-1 2^32 into its first product
#pragma unroll
  for (int k = 0; k < 16; ++k) a[(size_t)(j0 + TPC * k) * kRowLen] = x[k];
}

// One column job per CTA: grid (256 / 32 column blocks, rows).
template <int LOGN1>
__global__ void __launch_bounds__(2 << LOGN1, 1024 >> LOGN1) k_ntt_cols_fwd(uint32_t* __restrict__ data, RowMap rm, int r, int logN,
                                                             const uint2* __restrict__ tw,
                                                             const uint32_t* __restrict__ qtab) {
  __shared__ uint32_t s[(1 << LOGN1) * 32];
  cols_fwd_job<LOGN1>(data, rm, r, 1 << logN, blockIdx.x, blockIdx.y, threadIdx.x, s, tw, qtab);
}
template <int LOGN1>
__global__ void __launch_bounds__(2 << LOGN1, 1024 >> LOGN1) k_ntt_cols_inv(uint32_t* __restrict__ data, RowMap rm, int r, int logN,
                                                             const uint2* __restrict__ tw,
                                                             const uint32_t* __restrict__ qtab) {
  __shared__ uint32_t s[(1 << LOGN1) * 32];
  cols_inv_job<LOGN1>(data, rm, r, 1 << logN, blockIdx.x, blockIdx.y, threadIdx.x, s, tw, qtab);
}

// --------------------------------------------------------------- row pass
// The last 8 stages of the forward transform (first of the inverse) stay in
// one 256-word matrix row.  16 threads per row, 8 rows per CTA.  Layout A:
// thread j0 holds j0 + 16 k (distances 128 .. 16); layout B after a padded
// shared-memory exchange: 16 j0 + j (distances 8 .. 1), stored as four
// 128-bit writes.
constexpr int kRowsPerCta = 8;
__device__ __forceinline__ int rpad(int pos) { return pos + (pos >> 4); }

// Forward row pass on one matrix row held by 16 threads: x[k] = row[j0 + 16 k]
// on entry; on exit x[j] = row[16 j0 + j] of the transform, reduced to [0, q).
// sr: the row's padded shared-memory slot; the 16 threads are half a warp.
__device__ __forceinline__ void rows_fwd_core(uint32_t (&x)[16], int c, int j0, uint32_t* sr, int N,
                                              const uint2* __restrict__ w,
                                              uint32_t q) {
  // layout A: distance t = 16 h, stage index N/(2t), group c (8/h) + k/(2h)
#pragma unroll
  for (int h = 8; h >= 1; h >>= 1) {
    const int m = N / (32 * h);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      if (k & h) continue;
      const int i = c * (8 / h) + k / (2 * h);
      const uint2 t2 = __ldg(w + m + i);
      ct_bfly(x[k], x[k + h], t2.x, t2.y, q);
    }
  }
#pragma unroll
  for (int k = 0; k < 16; ++k) sr[rpad(j0 + 16 * k)] = x[k];
  __syncwarp();  // a row's 16 threads are half of one warp
#pragma unroll
  for (int j = 0; j < 16; ++j) x[j] = sr[rpad(16 * j0 + j)];
  // layout B: distance t = h, stage index N/(2h), group c (128/h) + j0 (8/h) + j/(2h)
#pragma unroll
  for (int h = 8; h >= 1; h >>= 1) {
    const int m = N / (2 * h);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if (j & h) continue;
      const int i = c * (128 / h) + j0 * (8 / h) + j / (2 * h);
      const uint2 t2 = __ldg(w + m + i);
      ct_bfly(x[j], x[j + h], t2.x, t2.y, q);
    }
  }
#pragma unroll
  for (int j = 0; j < 16; ++j) x[j] = reduce4(x[j], q);
}

__global__ void __launch_bounds__(16 * kRowsPerCta) k_ntt_rows_fwd(uint32_t* __restrict__ data, RowMap rm, int r,
                                                                   int logN, const uint2* __restrict__ tw,
                                                                   const uint32_t* __restrict__ qtab) {
  __shared__ uint32_t s[kRowsPerCta * (kRowLen + kRowLen / 16)];
  const int sub = threadIdx.x >> 4, j0 = threadIdx.x & 15;
  const int N = 1 << logN;
  const int p = rm.prime_of(blockIdx.y, r);
  const uint32_t q = __ldg(qtab + p);
  const int c = blockIdx.x * kRowsPerCta + sub;  // matrix row
  uint32_t* a = data + rm.row_of(blockIdx.y) * N + (size_t)c * kRowLen;
  uint32_t x[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) x[k] = a[j0 + 16 * k];
  rows_fwd_core(x, c, j0, s + sub * (kRowLen + kRowLen / 16), N, tw + (size_t)p * N, q);
  uint4* a4 = reinterpret_cast<uint4*>(a + 16 * j0);
#pragma unroll
  for (int v = 0; v < 4; ++v) a4[v] = make_uint4(x[4 * v], x[4 * v + 1], x[4 * v + 2], x[4 * v + 3]);
}

__global__ void __launch_bounds__(16 * kRowsPerCta) k_ntt_rows_inv(uint32_t* __restrict__ data, RowMap rm, int r,
                                                                   int logN, const uint2* __restrict__ tw,
                                                                   const uint32_t* __restrict__ qtab) {
  __shared__ uint32_t s[kRowsPerCta * (kRowLen + kRowLen / 16)];
  const int sub = threadIdx.x >> 4, j0 = threadIdx.x & 15;
  const int N = 1 << logN;
  const int p = rm.prime_of(blockIdx.y, r);
  const uint32_t q = __ldg(qtab + p);
  const uint2* w = tw + (size_t)p * N;
  const int c = blockIdx.x * kRowsPerCta + sub;
  uint32_t* a = data + rm.row_of(blockIdx.y) * N + (size_t)c * kRowLen;
  uint32_t* sr = s + sub * (kRowLen + kRowLen / 16);
  uint32_t x[16];
  const uint4* a4 = reinterpret_cast<const uint4*>(a + 16 * j0);
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const uint4 t = a4[v];
    x[4 * v] = t.x;
    x[4 * v + 1] = t.y;
    x[4 * v + 2] = t.z;
    x[4 * v + 3] = t.w;
  }
#pragma unroll
  for (int h = 1; h <= 8; h <<= 1) {
    const int m = N / (2 * h);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if (j & h) continue;
      const int i = c * (128 / h) + j0 * (8 / h) + j / (2 * h);
      const uint2 t2 = __ldg(w + m + i);
      gs_bfly(x[j], x[j + h], t2.x, t2.y, q);
    }
  }
#pragma unroll
  for (int j = 0; j < 16; ++j) sr[rpad(16 * j0 + j)] = x[j];
  __syncwarp();
#pragma unroll
  for (int k = 0; k < 16; ++k) x[k] = sr[rpad(j0 + 16 * k)];
#pragma unroll
  for (int h = 1; h <= 8; h <<= 1) {
    const int m = N / (32 * h);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      if (k & h) continue;
      const int i = c * (8 / h) + k / (2 * h);
      const uint2 t2 = __ldg(w + m + i);
      gs_bfly(x[k], x[k + h], t2.x, t2.y, q);
    }
  }
#pragma unroll
  for (int k = 0; k < 16; ++k) a[j0 + 16 * k] = x[k];
}

// ------------------------------------------------ fused transform-domain pass
// A ring product's forward row stages, its pointwise products and the inverse
// row stages of the results all work on the same 256-word matrix rows, so one
// kernel runs them back to back on registers: the products never go to
// memory in transform form.  16 threads per matrix row as in the row passes;
// a thread holds the same positions of every operand, so each twiddle pair is
// loaded once for all of them.  Exchange slots: one padded row per operand.
constexpr int kSlot = kRowLen + kRowLen / 16;

template <int R>
__device__ __forceinline__ void rows_fwd_multi(uint32_t (&x)[R][16], int c, int j0, uint32_t* sr, int N,
                                               const uint2* __restrict__ w,
                                               uint32_t q) {
#pragma unroll
  for (int h = 8; h >= 1; h >>= 1) {
    const int m = N / (32 * h);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      if (k & h) continue;
      const int i = c * (8 / h) + k / (2 * h);
      const uint2 t2 = __ldg(w + m + i);
      const uint32_t tw = t2.x, twp = t2.y;
#pragma unroll
      for (int o = 0; o < R; ++o) ct_bfly(x[o][k], x[o][k + h], tw, twp, q);
    }
  }
#pragma unroll
  for (int o = 0; o < R; ++o)
#pragma unroll
    for (int k = 0; k < 16; ++k) sr[o * kSlot + rpad(j0 + 16 * k)] = x[o][k];
  __syncwarp();
#pragma unroll
  for (int o = 0; o < R; ++o)
#pragma unroll
    for (int j = 0; j < 16; ++j) x[o][j] = sr[o * kSlot + rpad(16 * j0 + j)];
#pragma unroll
  for (int h = 8; h >= 1; h >>= 1) {
    const int m = N / (2 * h);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if (j & h) continue;
      const int i = c * (128 / h) + j0 * (8 / h) + j / (2 * h);
      const uint2 t2 = __ldg(w + m + i);
      const uint32_t tw = t2.x, twp = t2.y;
#pragma unroll
      for (int o = 0; o < R; ++o) ct_bfly(x[o][j], x[o][j + h], tw, twp, q);
    }
  }
}

// Inverse row stages: x[o][j] = row[16 j0 + j] in [0, 2q) on entry; on exit
// x[o][k] = row[j0 + 16 k], in [0, 2q), ready for the column stages.
template <int R>
__device__ __forceinline__ void rows_inv_multi(uint32_t (&x)[R][16], int c, int j0, uint32_t* sr, int N,
                                               const uint2* __restrict__ w,
                                               uint32_t q) {
#pragma unroll
  for (int h = 1; h <= 8; h <<= 1) {
    const int m = N / (2 * h);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if (j & h) continue;
      const int i = c * (128 / h) + j0 * (8 / h) + j / (2 * h);
      const uint2 t2 = __ldg(w + m + i);
      const uint32_t tw = t2.x, twp = t2.y;
#pragma unroll
      for (int o = 0; o < R; ++o) gs_bfly(x[o][j], x[o][j + h], tw, twp, q);
    }
  }
  __syncwarp();  // the forward exchange reads of this row are done
#pragma unroll
  for (int o = 0; o < R; ++o)
#pragma unroll
    for (int j = 0; j < 16; ++j) sr[o * kSlot + rpad(16 * j0 + j)] = x[o][j];
  __syncwarp();
#pragma unroll
  for (int o = 0; o < R; ++o)
#pragma unroll
    for (int k = 0; k < 16; ++k) x[o][k] = sr[o * kSlot + rpad(j0 + 16 * k)];
#pragma unroll
  for (int h = 1; h <= 8; h <<= 1) {
    const int m = N / (32 * h);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      if (k & h) continue;
      const int i = c * (8 / h) + k / (2 * h);
      const uint2 t2 = __ldg(w + m + i);
      const uint32_t tw = t2.x, twp = t2.y;
#pragma unroll
      for (int o = 0; o < R; ++o) gs_bfly(x[o][k], x[o][k + h], tw, twp, q);
    }
  }
}

// The row stages with a thread's twiddle pairs held in registers, so a loop over operands
// reuses them: t[0, 15) serve the layout-A stages (distance 16 h, h = 8, 4, 2, 1: 1, 2, 4, 8
// pairs, the group g of stage h at t[8 / h - 1 + g]), t[15, 30) the layout-B stages (distance h).
__device__ __forceinline__ void row_twiddles(uint2 (&t)[30], int c, int j0, int N, const uint2* __restrict__ w) {
#pragma unroll
  for (int h = 8; h >= 1; h >>= 1)
#pragma unroll
    for (int g = 0; g < 8 / h; ++g) t[8 / h - 1 + g] = __ldg(w + N / (32 * h) + c * (8 / h) + g);
#pragma unroll
  for (int h = 8; h >= 1; h >>= 1)
#pragma unroll
    for (int g = 0; g < 8 / h; ++g) t[15 + 8 / h - 1 + g] = __ldg(w + N / (2 * h) + c * (128 / h) + j0 * (8 / h) + g);
}
// Forward row stages of one row (as rows_fwd_multi<1>): x[k] = row[j0 + 16 k] in [0, 4q) on entry,
// x[j] = row[16 j0 + j] of the transform in [0, 4q) on exit; sr is the row's exchange slot.
__device__ __forceinline__ void rows_fwd_reg(uint32_t (&x)[16], int j0, uint32_t* sr, const uint2 (&t)[30],
                                             uint32_t q) {
#pragma unroll
  for (int h = 8; h >= 1; h >>= 1)
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      if (k & h) continue;
      const uint2 w = t[8 / h - 1 + k / (2 * h)];
      ct_bfly(x[k], x[k + h], w.x, w.y, q);
    }
#pragma unroll
  for (int k = 0; k < 16; ++k) sr[rpad(j0 + 16 * k)] = x[k];
  __syncwarp();
#pragma unroll
  for (int j = 0; j < 16; ++j) x[j] = sr[rpad(16 * j0 + j)];
#pragma unroll
  for (int h = 8; h >= 1; h >>= 1)
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if (j & h) continue;
      const uint2 w = t[15 + 8 / h - 1 + j / (2 * h)];
      ct_bfly(x[j], x[j + h], w.x, w.y, q);
    }
}
// Inverse row stages of one row (as rows_inv_multi<1>), with the inverse table's pairs in t.
__device__ __forceinline__ void rows_inv_reg(uint32_t (&x)[16], int j0, uint32_t* sr, const uint2 (&t)[30],
                                             uint32_t q) {
#pragma unroll
  for (int h = 1; h <= 8; h <<= 1)
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if (j & h) continue;
      const uint2 w = t[15 + 8 / h - 1 + j / (2 * h)];
      gs_bfly(x[j], x[j + h], w.x, w.y, q);
    }
#pragma unroll
  for (int j = 0; j < 16; ++j) sr[rpad(16 * j0 + j)] = x[j];
  __syncwarp();
#pragma unroll
  for (int k = 0; k < 16; ++k) x[k] = sr[rpad(j0 + 16 * k)];
#pragma unroll
  for (int h = 1; h <= 8; h <<= 1)
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      if (k & h) continue;
      const uint2 w = t[8 / h - 1 + k / (2 * h)];
      gs_bfly(x[k], x[k + h], w.x, w.y, q);
    }
}

// Tensor product in the transform domain (Sec. 5 pipeline): X = [batch][4][r][N]
// holds (B1, A1, B2, A2) after the forward column stages; the kernel finishes
// their transforms, forms D0 = B1 B2, D1 = A1 B2 + B1 A2, D2 = A1 A2
// (lazy Montgomery products; schoolbook, not Sec. 5's Karatsuba form: two
// reductions and four lazy products take fewer instructions than Karatsuba's
// three full products with four reductions, two modular additions and two
// modular subtractions) and runs the inverse row stages of D0, D1, D2 into
// blocks 0..2.
// The pass runs as loops: a thread loads its row's forward twiddle pairs once, transforms the
// four operand rows one after another (one copy of the stage code, not four interleaved copies)
// and parks each result in its exchange slot (B2, A2 reduced below q, so that B1, A1 in [0, 4q)
// can be the first operands: 4 q^2 < q 2^32); then, with the inverse pairs in the same
// registers, it forms each output from the slots and runs its inverse row stages.  D1 (which
// reads all four slots) goes first and exchanges in a fifth slot; D0 = B1 B2 then exchanges in
// B1's slot and D2 = A1 A2 in A1's, each after its own operands were read.  Against the
// four-operand unrolled form (one twiddle load per four butterflies, but four times the code)
// this keeps the pass out of instruction-fetch stalls: 7.20 -> 6.59 ms per N = 2^16 step of 64
// pairs.
// One job: matrix rows [8 bx, 8 bx + 8) of (ciphertext b, prime p), 128 threads, s holds
// kRowsPerCta * 5 * kSlot words.  Only warp-level synchronisation: each row's 16 threads own its slots.
__device__ __forceinline__ void rows_tensor_job(uint32_t* __restrict__ X, int r, int logN, int bx, int p, int b,
                                                uint32_t* s, const uint2* __restrict__ tw,
                                                const uint2* __restrict__ itw, const uint32_t* __restrict__ qtab,
                                                const uint32_t* __restrict__ qinv) {
  const int sub = threadIdx.x >> 4, j0 = threadIdx.x & 15;
  const int N = 1 << logN;
  const uint32_t q = __ldg(qtab + p), qi = __ldg(qinv + p);
  const size_t rowN = (size_t)r * N;
  const int c = bx * kRowsPerCta + sub;
  uint32_t* base = X + (size_t)b * 4 * rowN + (size_t)p * N + (size_t)c * kRowLen;
  uint32_t* sr = s + sub * 5 * kSlot;
  uint2 t[30];
  row_twiddles(t, c, j0, N, tw + (size_t)p * N);
#pragma unroll 1
  for (int o = 0; o < 4; ++o) {
    uint32_t x[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) x[k] = base[o * rowN + j0 + 16 * k];
    uint32_t* so = sr + o * kSlot;
    rows_fwd_reg(x, j0, so, t, q);
    __syncwarp();  // the row's exchange reads of this slot are done
    if (o < 2) {
#pragma unroll
      for (int j = 0; j < 16; ++j) so[rpad(16 * j0 + j)] = x[j];
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) so[rpad(16 * j0 + j)] = reduce4(x[j], q);
    }
  }
  row_twiddles(t, c, j0, N, itw + (size_t)p * N);
  __syncwarp();  // all four transformed rows are in their slots
#pragma unroll 1
  for (int o = 0; o < 3; ++o) {
    const int d = o == 0 ? 1 : 2 * (o - 1);  // output order D1, D0, D2
    uint32_t x[16];
    if (d == 1) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int pos = rpad(16 * j0 + j);
        const uint32_t v = mont_mul_lazy(sr[kSlot + pos], sr[2 * kSlot + pos], q, qi) +
                           mont_mul_lazy(sr[pos], sr[3 * kSlot + pos], q, qi);  // (0, 4q)
        x[j] = min(v, v - 2u * q);
      }
    } else {
      const uint32_t* u = sr + d * kSlot / 2;        // B1 (d = 0) or A1 (d = 2)
      const uint32_t* v = sr + (2 + d / 2) * kSlot;  // B2 or A2
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int pos = rpad(16 * j0 + j);
        x[j] = mont_mul_lazy(u[pos], v[pos], q, qi);
      }
    }
    uint32_t* ex = sr + (d == 1 ? 4 : d / 2) * kSlot;
    __syncwarp();  // the row's operand reads are done before its exchange slot is overwritten
    rows_inv_reg(x, j0, ex, t, q);
#pragma unroll
    for (int k = 0; k < 16; ++k) base[d * rowN + j0 + 16 * k] = x[k];
  }
}

// grid ((N / 256) / kRowsPerCta, batch * r); ciphertext fastest within a prime (L2 reuse of the
// prime's twiddles by consecutive CTAs).
__global__ void __launch_bounds__(16 * kRowsPerCta, 4) k_ntt_rows_tensor(uint32_t* __restrict__ X, int r, int logN,
                                                                        const uint2* __restrict__ tw,
                                                                        const uint2* __restrict__ itw,
                                                                        const uint32_t* __restrict__ qtab,
                                                                        const uint32_t* __restrict__ qinv) {
  __shared__ uint32_t s[kRowsPerCta * 5 * kSlot];
  const int nb = gridDim.y / r;
  const int p = blockIdx.y / nb, b = blockIdx.y - p * nb;
  rows_tensor_job(X, r, logN, blockIdx.x, p, b, s, tw, itw, qtab, qinv);
}

// The same pass with one operand per 16-thread group: a CTA takes 4 matrix rows of one
// (ciphertext, prime); group g (0..15) runs the forward row stages of operand g % 4 of row g / 4
// and leaves the transformed row in shared memory; after a barrier, group g < 12 forms output
// g % 3 of row g / 3 (D0 = B1 B2, D1 = A1 B2 + A2 B1, D2 = A1 A2, Montgomery) for its 16 positions
// and runs that output's inverse row stages (warps 6 and 7 sit out).  A thread's code covers one
// operand instead of four, which keeps the pass's instruction footprint small.
constexpr int kGRows = 4;  // matrix rows per CTA
__global__ void __launch_bounds__(256) k_ntt_rows_tensor_g(uint32_t* __restrict__ X, int r, int logN,
                                                           const uint2* __restrict__ tw,
                                                           const uint2* __restrict__ itw,
                                                           const uint32_t* __restrict__ qtab,
                                                           const uint32_t* __restrict__ qinv) {
  __shared__ uint32_t s[16 * kSlot];
  const int grp = threadIdx.x >> 4, j0 = threadIdx.x & 15;
  const int N = 1 << logN;
  const int nb = gridDim.y / r;
  const int p = blockIdx.y / nb, b = blockIdx.y - p * nb;
  const uint32_t q = __ldg(qtab + p), qi = __ldg(qinv + p);
  const size_t rowN = (size_t)r * N;
  uint32_t* base = X + (size_t)b * 4 * rowN + (size_t)p * N;
  {
    const int row = grp >> 2, op = grp & 3;
    const int c = blockIdx.x * kGRows + row;
    const uint32_t* a = base + op * rowN + (size_t)c * kRowLen;
    uint32_t x[1][16];
#pragma unroll
    for (int k = 0; k < 16; ++k) x[0][k] = a[j0 + 16 * k];
    uint32_t* sr = s + grp * kSlot;
    rows_fwd_multi<1>(x, c, j0, sr, N, tw + (size_t)p * N, q);
    __syncwarp();  // the exchange reads of this slot are done
#pragma unroll
    for (int j = 0; j < 16; ++j) sr[rpad(16 * j0 + j)] = reduce4(x[0][j], q);
  }
  __syncthreads();
  uint32_t y[1][16];
  int row = 0, o = 0;
  if (grp < 12) {
    row = grp / 3;
    o = grp - 3 * row;
    const uint32_t* B1 = s + (row * 4 + 0) * kSlot;
    const uint32_t* A1 = s + (row * 4 + 1) * kSlot;
    const uint32_t* B2 = s + (row * 4 + 2) * kSlot;
    const uint32_t* A2 = s + (row * 4 + 3) * kSlot;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int pos = rpad(16 * j0 + j);
      if (o == 0) {
        y[0][j] = mont_mul(B1[pos], B2[pos], q, qi);
      } else if (o == 2) {
        y[0][j] = mont_mul(A1[pos], A2[pos], q, qi);
      } else {
        y[0][j] = add_mod(mont_mul(A1[pos], B2[pos], q, qi), mont_mul(A2[pos], B1[pos], q, qi), q);
      }
    }
  }
  __syncthreads();  // every product read its operands: the slots are free for the inverse exchanges
  if (grp < 12) {
    const int c = blockIdx.x * kGRows + row;
    rows_inv_multi<1>(y, c, j0, s + grp * kSlot, N, itw + (size_t)p * N, q);
    uint32_t* d = base + o * rowN + (size_t)c * kRowLen;
#pragma unroll
    for (int k = 0; k < 16; ++k) d[j0 + 16 * k] = y[0][k];
  }
}

// Key product of a key switch (Sec. 6): Y = [batch][2][r][N] holds the lifted
// polynomial in block 0 after the forward column stages; the kernel finishes
// its transform, multiplies it by the key rows K[0][p], K[1][p] (transform
// form, Montgomery) and runs the inverse row stages of both products into
// blocks 0 and 1.
// One job: matrix rows [8 bx, 8 bx + 8) of (ciphertext b, prime p), 128 threads, s holds
// kRowsPerCta * 2 * kSlot words (warp-level synchronisation only).
__device__ __forceinline__ void rows_key_job(uint32_t* __restrict__ Y, const uint32_t* __restrict__ K, int krows,
                                             int r, int logN, int bx, int p, int b, uint32_t* s,
                                             const uint2* __restrict__ tw, const uint2* __restrict__ itw,
                                             const uint32_t* __restrict__ qtab,
                                             const uint32_t* __restrict__ qinv) {
  const int sub = threadIdx.x >> 4, j0 = threadIdx.x & 15;
  const int N = 1 << logN;
  const uint32_t q = __ldg(qtab + p), qi = __ldg(qinv + p);
  const int c = bx * kRowsPerCta + sub;
  const size_t coff = (size_t)c * kRowLen;
  uint32_t* y0 = Y + ((size_t)b * 2 * r + p) * N + coff;
  uint32_t* y1 = y0 + (size_t)r * N;
  uint32_t* sr = s + sub * 2 * kSlot;
  uint32_t x[2][16];
#pragma unroll
  for (int k = 0; k < 16; ++k) x[0][k] = y0[j0 + 16 * k];
  {
    uint32_t (&x0)[1][16] = *reinterpret_cast<uint32_t (*)[1][16]>(&x[0][0]);
    rows_fwd_multi<1>(x0, c, j0, sr, N, tw + (size_t)p * N, q);
  }
  // Montgomery products accept one operand in [0, 4q): 4 q^2 < q 2^32
  const uint4* kb = reinterpret_cast<const uint4*>(K + (size_t)p * N + coff + 16 * j0);
  const uint4* ka = reinterpret_cast<const uint4*>(K + (size_t)(krows + p) * N + coff + 16 * j0);
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const uint4 vb = __ldg(kb + v), va = __ldg(ka + v);
    const uint32_t kbv[4] = {vb.x, vb.y, vb.z, vb.w}, kav[4] = {va.x, va.y, va.z, va.w};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const uint32_t d = x[0][4 * v + u];
      x[0][4 * v + u] = mont_mul_lazy(d, kbv[u], q, qi);  // (0, 2q): what the inverse stages accept
      x[1][4 * v + u] = mont_mul_lazy(d, kav[u], q, qi);
    }
  }
  rows_inv_multi<2>(x, c, j0, sr, N, itw + (size_t)p * N, q);
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    y0[j0 + 16 * k] = x[0][k];
    y1[j0 + 16 * k] = x[1][k];
  }
}

__global__ void __launch_bounds__(16 * kRowsPerCta) k_ntt_rows_key(uint32_t* __restrict__ Y,
                                                                   const uint32_t* __restrict__ K, int krows, int r,
                                                                   int logN, const uint2* __restrict__ tw,
                                                                   const uint2* __restrict__ itw,
                                                                   const uint32_t* __restrict__ qtab,
                                                                   const uint32_t* __restrict__ qinv) {
  __shared__ uint32_t s[kRowsPerCta * 2 * kSlot];
  // ciphertext fastest within a prime: consecutive CTAs reuse the prime's twiddles (and key rows) from L2
  const int nb = gridDim.y / r;
  const int p = blockIdx.y / nb, b = blockIdx.y - p * nb;
  rows_key_job(Y, K, krows, r, logN, blockIdx.x, p, b, s, tw, itw, qtab, qinv);
}

// ------------------------------------------- automorphism in the transform domain
// kappa_g: a(X) -> a(X^g) (Sec. 6 leftrotate with g = 5^j, conjugate with g = 2N - 1).  The forward
// transform leaves a(psi^(2 brv(k) + 1)) at index k, so
//   NTT(kappa_g a)[k] = NTT(a)[pi(k)],  pi(k) = brv((g brv(k) + (g - 1)/2) mod N)
// (brv over log N bits).  With k = 256 c + m (matrix row c, column m), brv(k) = brv8(m) N1 + brv(c)
// (N1 = N / 256), so every output row c reads one source row c' = brv(w mod N1),
// w = (g brv(c) + (g - 1)/2) mod N, at columns m' = brv8((w / N1 + g brv8(m)) mod 256).  A rotation
// by many steps therefore lifts and transforms its input once and applies each kappa_g as a row
// gather in front of the key products.
__device__ __forceinline__ uint32_t brv_bits(uint32_t x, int bits) { return bits ? __brev(x) >> (32 - bits) : 0u; }

// Fused: for matrix row c of (ciphertext b, prime p), gather row c' of AH (the forward transform
// of the key-switch input, [batch][r][N]), multiply by the key rows K[0][p], K[1][p] (Montgomery)
// and run the inverse row stages of both products into Y = [batch][2][r][N] blocks 0 and 1.
__global__ void __launch_bounds__(16 * kRowsPerCta) k_ntt_rows_key_perm(uint32_t* __restrict__ Y,
                                                                        const uint32_t* __restrict__ AH,
                                                                        const uint32_t* __restrict__ K, int krows,
                                                                        int r, int logN, uint32_t g,
                                                                        const uint2* __restrict__ itw,
                                                                        const uint32_t* __restrict__ qtab,
                                                                        const uint32_t* __restrict__ qinv) {
  __shared__ uint32_t s[kRowsPerCta * 2 * kSlot];
  const int sub = threadIdx.x >> 4, j0 = threadIdx.x & 15;
  const int N = 1 << logN, logN1 = logN - 8, N1 = 1 << logN1;
  const int nb = gridDim.y / r;
  const int p = blockIdx.y / nb, b = blockIdx.y - p * nb;
  const uint32_t q = __ldg(qtab + p), qi = __ldg(qinv + p);
  const int c = blockIdx.x * kRowsPerCta + sub;
  const uint32_t w = (g * brv_bits((uint32_t)c, logN1) + (g - 1u) / 2u) & (uint32_t)(N - 1);
  const int cs = (int)brv_bits(w & (uint32_t)(N1 - 1), logN1);
  const uint32_t whi = w >> logN1;
  uint32_t* sr = s + sub * 2 * kSlot;
  const uint32_t* src = AH + ((size_t)b * r + p) * N + (size_t)cs * kRowLen;
#pragma unroll
  for (int k = 0; k < 16; ++k) sr[j0 + 16 * k] = __ldg(src + j0 + 16 * k);
  __syncwarp();
  const size_t coff = (size_t)c * kRowLen;
  const uint4* kb = reinterpret_cast<const uint4*>(K + (size_t)p * N + coff + 16 * j0);
  const uint4* ka = reinterpret_cast<const uint4*>(K + (size_t)(krows + p) * N + coff + 16 * j0);
  uint32_t x[2][16];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const uint4 vb = __ldg(kb + v), va = __ldg(ka + v);
    const uint32_t kbv[4] = {vb.x, vb.y, vb.z, vb.w}, kav[4] = {va.x, va.y, va.z, va.w};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const uint32_t m = 16u * j0 + 4u * v + u;
      const uint32_t mp = brv_bits((whi + g * brv_bits(m, 8)) & 255u, 8);
      const uint32_t d = sr[mp];
      x[0][4 * v + u] = mont_mul_lazy(d, kbv[u], q, qi);
      x[1][4 * v + u] = mont_mul_lazy(d, kav[u], q, qi);
    }
  }
  rows_inv_multi<2>(x, c, j0, sr, N, itw + (size_t)p * N, q);  // syncs the warp before reusing sr
  uint32_t* y0 = Y + ((size_t)b * 2 * r + p) * N + coff;
  uint32_t* y1 = y0 + (size_t)r * N;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    y0[j0 + 16 * k] = x[0][k];
    y1[j0 + 16 * k] = x[1][k];
  }
}

// Any ring size: the same gather and key products, one thread per transform coefficient
// (the inverse transforms follow as a separate launch).  grid (N / 256, batch * r).
__global__ void k_pw_key_perm(uint32_t* __restrict__ Y, const uint32_t* __restrict__ AH,
                              const uint32_t* __restrict__ K, int krows, int r, int logN, uint32_t g,
                              const uint32_t* __restrict__ qtab, const uint32_t* __restrict__ qinv) {
  const int N = 1 << logN;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const int p = blockIdx.y % r, b = blockIdx.y / r;
  const uint32_t q = __ldg(qtab + p), qi = __ldg(qinv + p);
  const uint32_t u = (uint32_t)(((uint64_t)g * brv_bits((uint32_t)k, logN) + (g - 1u) / 2u) & (uint64_t)(N - 1));
  const uint32_t d = __ldg(AH + ((size_t)b * r + p) * N + brv_bits(u, logN));
  uint32_t* y0 = Y + ((size_t)b * 2 * r + p) * N;
  y0[k] = mont_mul(d, __ldg(K + (size_t)p * N + k), q, qi);
  y0[(size_t)r * N + k] = mont_mul(d, __ldg(K + (size_t)(krows + p) * N + k), q, qi);
}

static int ntt_chunk(const fhe_ctx* ctx, uint32_t* data, RowMap rm, int rows, int r, bool inverse,
                     cudaStream_t st) {
  const int logN = ctx->prm.logN, N = ctx->N;
  const uint2* tw = inverse ? ctx->d_ipsi2 : ctx->d_psi2;
  ProfScope ps(ctx, inverse ? FHE_K_NTT_INV : FHE_K_NTT_FWD, logN <= 12 ? 1 : 2, st);
  if (logN <= 12) {
    const int threads = N / 2 < 32 ? 32 : (N / 2 > 512 ? 512 : N / 2);
    const size_t smem = (size_t)N * 4;
    if (inverse)
      k_ntt_small<true><<<rows, threads, smem, st>>>(data, rm, r, logN, tw, ctx->d_q);
    else
      k_ntt_small<false><<<rows, threads, smem, st>>>(data, rm, r, logN, tw, ctx->d_q);
    return FHE_OK;
  }
  const int logN1 = logN - 8, N1 = 1 << logN1;
  dim3 gcols(kRowLen / 32, rows), grows(N1 / kRowsPerCta, rows);
#define FHE_NTT_COLS(L)                                                                                    \
  case L:                                                                                                  \
    if (inverse)                                                                                           \
      k_ntt_cols_inv<L><<<gcols, 2 << L, 0, st>>>(data, rm, r, logN, tw, ctx->d_q);                                       \
    else                                                                                                   \
      k_ntt_cols_fwd<L><<<gcols, 2 << L, 0, st>>>(data, rm, r, logN, tw, ctx->d_q);                   \
    break;
  if (!inverse) {
    switch (logN1) { FHE_NTT_COLS(5) FHE_NTT_COLS(6) FHE_NTT_COLS(7) FHE_NTT_COLS(8) }
    k_ntt_rows_fwd<<<grows, 16 * kRowsPerCta, 0, st>>>(data, rm, r, logN, tw, ctx->d_q);
  } else {
    k_ntt_rows_inv<<<grows, 16 * kRowsPerCta, 0, st>>>(data, rm, r, logN, tw, ctx->d_q);
    switch (logN1) { FHE_NTT_COLS(5) FHE_NTT_COLS(6) FHE_NTT_COLS(7) FHE_NTT_COLS(8) }
  }
#undef FHE_NTT_COLS
  return FHE_OK;
}

static void cols_launch(const fhe_ctx* ctx, uint32_t* data, RowMap rm, int rows, int r, bool inverse,
                        cudaStream_t st) {
  const int logN = ctx->prm.logN, logN1 = logN - 8;
  dim3 g(kRowLen / 32, rows);
#define FHE_NTT_COLS_ONLY(L)                                                                                 \
  case L:                                                                                                    \
    if (inverse)                                                                                             \
      k_ntt_cols_inv<L><<<g, 2 << L, 0, st>>>(data, rm, r, logN, ctx->d_ipsi2, ctx->d_q);                              \
    else                                                                                                     \
      k_ntt_cols_fwd<L><<<g, 2 << L, 0, st>>>(data, rm, r, logN, ctx->d_psi2, ctx->d_q);       \
    break;
  switch (logN1) { FHE_NTT_COLS_ONLY(5) FHE_NTT_COLS_ONLY(6) FHE_NTT_COLS_ONLY(7) FHE_NTT_COLS_ONLY(8) }
#undef FHE_NTT_COLS_ONLY
}

int launch_ring_tensor(const fhe_ctx* ctx, uint32_t* X, int r, int nbatch, cudaStream_t st) {
  const int logN = ctx->prm.logN, N = ctx->N;
  if (logN <= 12 || (size_t)nbatch * 4 * r > 65535u || ctx->ntt_form == FHE_NTT_SPLIT) {
    int rc = launch_ntt(ctx, X, nbatch * 4, r, r, r, false, st);
    if (!rc) rc = launch_pointwise_tensor(ctx, X, r, nbatch, st);
    return rc ? rc : launch_ntt(ctx, X, nbatch, 3 * r, 4 * r, r, true, st);
  }
  {
    ProfScope ps(ctx, FHE_K_NTT_FWD, 1, st);
    cols_launch(ctx, X, RowMap{r, r}, nbatch * 4 * r, r, false, st);
  }
  {
    ProfScope ps(ctx, FHE_K_NTT_PW, 1, st);
    if (ctx->ntt_form == FHE_NTT_FUSED_GROUPS) {
      dim3 grid((N >> 8) / kGRows, nbatch * r);
      k_ntt_rows_tensor_g<<<grid, 256, 0, st>>>(X, r, logN, ctx->d_psi2, ctx->d_ipsi2, ctx->d_q, ctx->d_qinv);
    } else {
      dim3 grid((N >> 8) / kRowsPerCta, nbatch * r);
      k_ntt_rows_tensor<<<grid, 16 * kRowsPerCta, 0, st>>>(X, r, logN, ctx->d_psi2, ctx->d_ipsi2, ctx->d_q,
                                                             ctx->d_qinv);
    }
  }
  {
    ProfScope ps(ctx, FHE_K_NTT_INV, 1, st);
    cols_launch(ctx, X, RowMap{3 * r, 4 * r}, nbatch * 3 * r, r, true, st);
  }
  return FHE_OK;
}

int launch_ring_key(const fhe_ctx* ctx, uint32_t* Y, const uint32_t* K, int krows, int r, int nbatch,
                    cudaStream_t st) {
  const int logN = ctx->prm.logN, N = ctx->N;
  if (r > krows) return FHE_EINVAL;
  if (logN <= 12 || (size_t)nbatch * 2 * r > 65535u || ctx->ntt_form == FHE_NTT_SPLIT) {
    int rc = launch_ntt(ctx, Y, nbatch, r, 2 * r, r, false, st);
    if (!rc) rc = launch_pointwise_key(ctx, Y, K, krows, r, nbatch, st);
    return rc ? rc : launch_ntt(ctx, Y, nbatch * 2, r, r, r, true, st);
  }
  {
    ProfScope ps(ctx, FHE_K_NTT_FWD, 1, st);
    cols_launch(ctx, Y, RowMap{r, 2 * r}, nbatch * r, r, false, st);
  }
  {
    ProfScope ps(ctx, FHE_K_NTT_PW, 1, st);
    dim3 grid((N >> 8) / kRowsPerCta, nbatch * r);
    k_ntt_rows_key<<<grid, 16 * kRowsPerCta, 0, st>>>(Y, K, krows, r, logN, ctx->d_psi2, ctx->d_ipsi2, ctx->d_q,
                                                      ctx->d_qinv);
  }
  {
    ProfScope ps(ctx, FHE_K_NTT_INV, 1, st);
    cols_launch(ctx, Y, RowMap{r, r}, nbatch * 2 * r, r, true, st);
  }
  return FHE_OK;
}

int launch_key_perm(const fhe_ctx* ctx, const uint32_t* AH, uint32_t* Y, const uint32_t* K, int krows, int r,
                    int nbatch, uint32_t g, cudaStream_t st) {
  const int logN = ctx->prm.logN, N = ctx->N;
  if (r > krows || r < 1 || nbatch < 1 || !(g & 1u) || g >= 2u * (uint32_t)N) {
    set_error("key_perm: bad arguments (r %d, key rows %d, g %u)", r, krows, g);
    return FHE_EINVAL;
  }
  if (logN <= 12 || (size_t)nbatch * r > 65535u || ctx->ntt_form == FHE_NTT_SPLIT) {
    if ((size_t)nbatch * r > 65535u) {
      set_error("key_perm: %d x %d rows exceed one launch", nbatch, r);
      return FHE_EINVAL;
    }
    {
      ProfScope ps(ctx, FHE_K_POINTWISE, 1, st);
      const int threads = N < 256 ? N : 256;
      k_pw_key_perm<<<dim3((N + threads - 1) / threads, nbatch * r), threads, 0, st>>>(Y, AH, K, krows, r, logN, g,
                                                                                    ctx->d_q, ctx->d_qinv);
    }
    return launch_ntt(ctx, Y, nbatch * 2, r, r, r, true, st);
  }
  {
    ProfScope ps(ctx, FHE_K_NTT_PW, 1, st);
    dim3 grid((N >> 8) / kRowsPerCta, nbatch * r);
    k_ntt_rows_key_perm<<<grid, 16 * kRowsPerCta, 0, st>>>(Y, AH, K, krows, r, logN, g, ctx->d_ipsi2, ctx->d_q,
                                                           ctx->d_qinv);
  }
  {
    ProfScope ps(ctx, FHE_K_NTT_INV, 1, st);
    cols_launch(ctx, Y, RowMap{r, r}, nbatch * 2 * r, r, true, st);
  }
  return FHE_OK;
}

// ------------------------------------------------------------ work-table launches
// One launch runs a transform stage of many ring products of different ring sizes and prime counts
// (a batch of groups, NttTable).  A CTA takes units u = blockIdx.x, blockIdx.x + gridDim.x, ...; the
// segment of its first unit is found by a binary search of the segments' first units, later ones by
// a forward scan from there (u only grows).
__device__ __forceinline__ int table_seg_first(const NttTable& t, int u) {
  int lo = 0, hi = t.nseg - 1;  // the last segment whose first unit is <= u
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (t.seg[mid].unit0 <= u)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}
__device__ __forceinline__ int table_seg(const NttTable& t, int u, int si) {
  if (si < 0) return table_seg_first(t, u);
  while (si + 1 < t.nseg && u >= t.seg[si + 1].unit0) ++si;
  return si;
}

// Column stages of rows [y0, y1) of a segment with N1 = 2^LOGN1: (y1 - y0) * 8 column jobs of
// 2 N1 threads, 256 / N1 of them side by side in the CTA's 512 threads per round (every round is
// full: 256 / N1 divides 8).  The barrier after a round frees the shared memory for the next.
template <int LOGN1, bool INV>
__device__ __forceinline__ void cols_table_rows(const NttSeg& g, int y0, int y1, uint32_t* s) {
  constexpr int T = 2 << LOGN1, P = 512 / T;
  const int sub = threadIdx.x / T, tid = threadIdx.x % T;
  const RowMap rm{g.group_rows, g.group_stride};
  const int N = 1 << g.logN;
  uint32_t* ss = s + sub * (T / 2) * 32;
  for (int j = y0 * 8 + sub; j < y1 * 8; j += P) {
    if (INV)
      cols_inv_job<LOGN1>(g.data, rm, g.r, N, j & 7, j >> 3, tid, ss, g.tw, g.q);
    else
      cols_fwd_job<LOGN1>(g.data, rm, g.r, N, j & 7, j >> 3, tid, ss, g.tw, g.q);
    __syncthreads();
  }
}

template <int LOGN1, bool INV>
__device__ __forceinline__ void cols_table_unit(const NttTable& t, int u, int si, uint32_t* s) {
  const NttSeg& g = t.seg[si];
  const int y0 = (u - g.unit0) * t.unit_rows;
  cols_table_rows<LOGN1, INV>(g, y0, min(y0 + t.unit_rows, g.rows), s);
}

// Persistent: a grid of a few CTAs per SM walks the units (40 registers, 3 CTAs of 512 threads per SM).
template <bool INV>
__global__ void __launch_bounds__(512, 3) k_ntt_cols_table(const __grid_constant__ NttTable t) {
  __shared__ uint32_t s[256 * 32];
  int si = -1;
  for (int u = blockIdx.x; u < t.total; u += gridDim.x) {
    si = table_seg(t, u, si);
    switch (t.seg[si].logN) {
      case 13: cols_table_unit<5, INV>(t, u, si, s); break;
      case 14: cols_table_unit<6, INV>(t, u, si, s); break;
      case 15: cols_table_unit<7, INV>(t, u, si, s); break;
      default: cols_table_unit<8, INV>(t, u, si, s); break;
    }
  }
}
// One round per CTA: unit u of a segment is the 256 / N1 column jobs u (256 / N1) .. of its rows (no
// loop, 4 CTAs of 512 threads per SM as the one-group kernels).
template <int LOGN1, bool INV>
__device__ __forceinline__ void cols_table_round(const NttSeg& g, int v, uint32_t* s) {
  constexpr int T = 2 << LOGN1, P = 512 / T;
  const int sub = threadIdx.x / T, j = v * P + sub;
  const RowMap rm{g.group_rows, g.group_stride};
  uint32_t* ss = s + sub * (T / 2) * 32;
  if (INV)
    cols_inv_job<LOGN1>(g.data, rm, g.r, 1 << g.logN, j & 7, j >> 3, threadIdx.x % T, ss, g.tw, g.q);
  else
    cols_fwd_job<LOGN1>(g.data, rm, g.r, 1 << g.logN, j & 7, j >> 3, threadIdx.x % T, ss, g.tw, g.q);
}
template <bool INV>
__global__ void __launch_bounds__(512, 4) k_ntt_cols_table1(const __grid_constant__ NttTable t) {
  __shared__ uint32_t s[256 * 32];
  const int si = table_seg_first(t, blockIdx.x);
  const NttSeg& g = t.seg[si];
  const int v = blockIdx.x - g.unit0;
  switch (g.logN) {
    case 13: cols_table_round<5, INV>(g, v, s); break;
    case 14: cols_table_round<6, INV>(g, v, s); break;
    case 15: cols_table_round<7, INV>(g, v, s); break;
    default: cols_table_round<8, INV>(g, v, s); break;
  }
}

// Fused row passes: unit v of a segment = row block v mod (N / 2048) of by = v / (N / 2048), with
// prime p = by / nb and ciphertext b = by mod nb (ciphertext fastest within a prime, as in the
// one-group kernels).  A row's 16 threads own its exchange slots; the warp barrier after a unit
// orders its last slot reads before the next unit's first writes.
__global__ void __launch_bounds__(16 * kRowsPerCta, 4) k_ntt_rows_tensor_table(const __grid_constant__ NttTable t) {
  __shared__ uint32_t s[kRowsPerCta * 5 * kSlot];
  int si = -1;
  for (int u = blockIdx.x; u < t.total; u += gridDim.x) {
    si = table_seg(t, u, si);
    const NttSeg& g = t.seg[si];
    const int v = u - g.unit0, lb = g.logN - 11;
    const int by = v >> lb, p = by / g.nb;
    rows_tensor_job(g.data, g.r, g.logN, v & ((1 << lb) - 1), p, by - p * g.nb, s, g.tw, g.itw, g.q, g.qinv);
    __syncwarp();
  }
}

__global__ void __launch_bounds__(16 * kRowsPerCta) k_ntt_rows_key_table(const __grid_constant__ NttTable t) {
  __shared__ uint32_t s[kRowsPerCta * 2 * kSlot];
  int si = -1;
  for (int u = blockIdx.x; u < t.total; u += gridDim.x) {
    si = table_seg(t, u, si);
    const NttSeg& g = t.seg[si];
    const int v = u - g.unit0, lb = g.logN - 11;
    const int by = v >> lb, p = by / g.nb;
    rows_key_job(g.data, g.key, g.krows, g.r, g.logN, v & ((1 << lb) - 1), p, by - p * g.nb, s, g.tw, g.itw, g.q,
                 g.qinv);
    __syncwarp();
  }
}

int launch_ntt_table(const fhe_ctx* prof_ctx, NttTable& t, int stage, int ctas_per_sm, cudaStream_t st) {
  if (t.nseg < 1 || t.nseg > kTableSegs || stage < kTableColsFwd || stage > kTableRowsKey || ctas_per_sm < 0 ||
      t.unit_rows < 1) {
    set_error("ntt_table: bad table (%d segments, stage %d)", t.nseg, stage);
    return FHE_EINVAL;
  }
  const bool cols = stage == kTableColsFwd || stage == kTableColsInv;
  long long total = 0;
  for (int i = 0; i < t.nseg; ++i) {
    NttSeg& g = t.seg[i];
    if (g.logN < 13 || g.logN > 16 || !g.data || !g.tw || !g.q || g.r < 1 || g.nb < 1 ||
        (cols && (g.rows < 1 || g.group_rows < 1 || g.group_stride < g.group_rows)) ||
        (!cols && (!g.itw || !g.qinv)) || (stage == kTableRowsKey && (!g.key || g.krows < g.r))) {
      set_error("ntt_table: segment %d malformed", i);
      return FHE_EINVAL;
    }
    // columns, one CTA per unit: a unit is one round of 256 / N1 jobs (rows * 8 jobs in all)
    const long long units = cols ? (ctas_per_sm == 0 ? ((long long)g.rows * 8) >> (16 - g.logN)
                                                     : (g.rows + t.unit_rows - 1) / t.unit_rows)
                                 : ((long long)g.nb * g.r) << (g.logN - 11);
    g.unit0 = (int)total;
    g.units = (int)units;
    total += units;
    if (total > 0x7fffffffLL) {
      set_error("ntt_table: %lld units exceed one launch", total);
      return FHE_EINVAL;
    }
  }
  t.total = (int)total;
  int dev = 0, nsm = 0, fit = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const bool one = ctas_per_sm == 0;  // columns: the loop-free kernel, one CTA per unit
  const void* fn = stage == kTableColsFwd   ? (one ? (const void*)k_ntt_cols_table1<false>
                                                   : (const void*)k_ntt_cols_table<false>)
                   : stage == kTableColsInv ? (one ? (const void*)k_ntt_cols_table1<true>
                                                   : (const void*)k_ntt_cols_table<true>)
                   : stage == kTableRowsTensor ? (const void*)k_ntt_rows_tensor_table
                                               : (const void*)k_ntt_rows_key_table;
  const int threads = cols ? 512 : 16 * kRowsPerCta;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, fn, threads, 0);
  if (e != cudaSuccess) {
    set_error("ntt_table: %s", cudaGetErrorString(e));
    return FHE_ECUDA;
  }
  long long grid = total;
  if (ctas_per_sm > 0) {
    const long long per = ctas_per_sm < fit ? ctas_per_sm : (fit > 0 ? fit : 1);
    grid = (long long)nsm * per < total ? (long long)nsm * per : total;
  }
  const int kclass = stage == kTableColsFwd ? FHE_K_NTT_FWD : stage == kTableColsInv ? FHE_K_NTT_INV : FHE_K_NTT_PW;
  ProfScope ps(prof_ctx, kclass, 1, st);
  switch (stage) {
    case kTableColsFwd:
      if (one)
        k_ntt_cols_table1<false><<<(unsigned)grid, 512, 0, st>>>(t);
      else
        k_ntt_cols_table<false><<<(unsigned)grid, 512, 0, st>>>(t);
      break;
    case kTableColsInv:
      if (one)
        k_ntt_cols_table1<true><<<(unsigned)grid, 512, 0, st>>>(t);
      else
        k_ntt_cols_table<true><<<(unsigned)grid, 512, 0, st>>>(t);
      break;
    case kTableRowsTensor: k_ntt_rows_tensor_table<<<(unsigned)grid, 16 * kRowsPerCta, 0, st>>>(t); break;
    default: k_ntt_rows_key_table<<<(unsigned)grid, 16 * kRowsPerCta, 0, st>>>(t); break;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("ntt_table: launch failed: %s", cudaGetErrorString(e));
    return FHE_ECUDA;
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
