// FP64-accurate Nystrom sketch Y = G Omega = J^T diag(w) (J Omega) (App. A, the sketch step) on
// the tcgen05 tensor cores, for an FP32 Jacobian.
//
// Method: an error-free split of the operands into BF16 "digit planes" (the splitting idea of
// Ozaki, Ogita, Oishi and Rump, "Error-free transformations of matrix multiplication by using
// fast routines of matrix multiplication and its applications", Numer. Algorithms 59 (2012),
// here with signed base-256 digits and exact fixed-point accumulation):
//   * each row n of J is scaled by a power of two 2^-e_n (e_n: max_k |J_nk| < 2^e_n) and written
//     as J_nk = 2^(e_n - 7) (a_0 + a_1 2^-8 + ... + a_4 2^-32) with integer digits |a_s| <= 128
//     (round-to-nearest digits: each next digit takes the rounding remainder times 256);
//   * each column j of Omega likewise with 5 digits (exact for every entry above 2^-16 of its
//     column's largest; below that, truncated at 2^-41 of it);
//   * Z'' = diag(w) diag(2^e_n) (J Omega) is split per column with 6 digits;
//   * digit s is stored as the BF16 number a_s 2^(-8 s) (exact: 8 significant bits), so a product
//     of digit planes s and t carries its weight 2^(-8 (s + t)) by itself.
// GEMM1 Z = J Omega and GEMM2 Y = J^T Z'' then become sums over digit-plane products (s, t) with
// s + t <= 5 ("levels"; the dropped levels weigh <= 2^-48 of the leading one).  Levels 0 to 3
// are summed exactly, each in its own accumulator: within one level every product is an integer
// times the level's weight, a K-chunk of 256 keeps every partial sum within 2^24 such units (at
// most 4 pairs x 256 x 2^14), and the tensor core's FP32 accumulation of such sums is exact
// (measured on GB300 with integer digit data up to 2^24: no rounding; mixed magnitudes inside one
// 16-wide group, or an accumulator of a larger magnitude than its addends, do round, which the
// split avoids by giving every MMA a single (s, t) pair and every exact level its own
// accumulator).  Levels 4 and 5 (weight <= 2^-32) share a fifth FP32 accumulator, whose rounding
// (half a level-4 unit per addition) stays below 2^-52 of the leading level.  Each CTA sums one
// 128 x 96 output tile over one K-chunk into the five TMEM accumulators (480 of 512 columns),
// combines them into a double-float value, and writes it as a split-K partial; a second kernel
// adds the partials of a tile in a fixed order (deterministic) and applies the power-of-two scales.
//
// Kernel structure (k_oz_gemm): warp 0 lane 0 issues TMA loads of digit tiles (A: 128 rows, 16 KB;
// B: 96 rows, 12 KB; 64 BF16 = 128 bytes per row, 128-byte swizzle) into two shared-memory rings
// (OzSmem); per 64-wide k-block, the B digit tiles (descending digit) and then the A digit tiles
// (ascending digit).  Warp 1 lane 0 issues tcgen05.mma (kind::f16, M = 128, N = 96, K = 16) pair
// by pair, each k-block in straight-line code, and releases each tile after its last use.  Warps
// 2..17 (four per TMEM lane quarter) drain the accumulators with tcgen05.ld.  Waits follow the
// bounded protocol of tc_common.cuh.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <new>

#include "df.cuh"
#include "ngd_internal.cuh"
#include "sketch_oz.cuh"
#include "tc_common.cuh"

namespace ngd {

namespace {

using namespace tc;

constexpr int kDigJ = 5;       // digits of the row-scaled Jacobian
constexpr int kDigOm = 5;      // digits of the column-scaled test matrix
constexpr int kDigZ = 6;       // digits of the column-scaled Z''
constexpr int kLevels = 5;     // pairs (s, t) with s + t <= kLevels are kept
constexpr int kChunk = 256;    // K per CTA: exact level sums (4 pairs x 256 x 2^14 = 2^24)
constexpr int kBM = 128, kBN = 96, kBK = 64;
constexpr int kTile = kBM * kBK * 2;                        // 16 KB slot: 128 rows x 128 bytes
constexpr int kTileB = kBN * kBK * 2;                       // 12 KB of a B tile
constexpr int kAcc = 5;                                     // TMEM accumulators of kBN columns
constexpr size_t kPartialCap = size_t(1) << 30;             // bytes of split-K partials per launch

int64_t rup(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// exponent e with m < 2^e (m >= 0; 0 for m = 0)
__device__ __forceinline__ int exp_above(float m) {
  int e = 0;
  frexpf(m, &e);
  return m > 0.0f ? e : 0;
}
__device__ __forceinline__ int exp_above_d(double m) {
  int e = 0;
  frexp(m, &e);
  return m > 0.0 ? e : 0;
}

// ---------------------------------------------------------------------------- splits
// e_n of every row of J (max over the row's p entries; padding columns are zero).  One warp per row.
__global__ void k_oz_rowexp(const float* __restrict__ J, int64_t ldJ, int64_t N, int* __restrict__ jexp) {
  const int64_t n = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (n >= N) return;
  const float4* row = reinterpret_cast<const float4*>(J + n * ldJ);
  float m = 0.0f;
  for (int64_t i = lane; i < ldJ / 4; i += 32) {
    const float4 v = row[i];
    m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) jexp[n] = exp_above(m);
}

// Digit planes of the row-scaled J in both layouts: JD[s] (N x ldJ, as J) for Z = J Omega and
// JDT[s] (ldJ x ldN, transposed; rows n >= N zero) for Y = J^T Z''.  32 x 32 tiles.
__global__ void k_oz_split_rows(const float* __restrict__ J, int64_t ldJ, int64_t N, const int* __restrict__ jexp,
                                __nv_bfloat16* __restrict__ JD, __nv_bfloat16* __restrict__ JDT, int64_t ldN) {
  __shared__ __nv_bfloat16 tile[kDigJ][32][34];
  const int64_t k0 = (int64_t)blockIdx.x * 32, n0 = (int64_t)blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int i = ty; i < 32; i += blockDim.y) {
    const int64_t n = n0 + i, k = k0 + tx;
    float a[kDigJ];
    if (n < N) {
      float r = ldexpf(J[n * ldJ + k], 7 - jexp[n]);      // |r| < 128
#pragma unroll
      for (int s = 0; s < kDigJ; ++s) {
        a[s] = rintf(r);
        r = (r - a[s]) * 256.0f;                            // exact
      }
    } else {
#pragma unroll
      for (int s = 0; s < kDigJ; ++s) a[s] = 0.0f;
    }
#pragma unroll
    for (int s = 0; s < kDigJ; ++s) {
      const __nv_bfloat16 b = __float2bfloat16_rn(ldexpf(a[s], -8 * s));   // exact
      tile[s][i][tx] = b;
      if (n < N) JD[(int64_t)s * N * ldJ + n * ldJ + k] = b;
    }
  }
  __syncthreads();
  for (int i = ty; i < 32; i += blockDim.y) {
    const int64_t k = k0 + i, n = n0 + tx;
#pragma unroll
    for (int s = 0; s < kDigJ; ++s) JDT[(int64_t)s * ldJ * ldN + k * ldN + n] = tile[s][tx][i];
  }
}

// Column exponents of a column-major matrix V (rows x cols, leading dimension ld): one block per
// column; the maximum taken on the magnitudes' bit patterns (non-negative floats order as their
// bits) in the integer pipes.
template <typename T>
__global__ void k_oz_colexp(const T* __restrict__ V, int64_t ld, int64_t rows, int* __restrict__ cexp) {
  using U = typename std::conditional<sizeof(T) == 4, unsigned, unsigned long long>::type;
  constexpr U kAbs = sizeof(T) == 4 ? (U)0x7fffffffu : (U)0x7fffffffffffffffull;
  __shared__ U red[32];
  const U* col = reinterpret_cast<const U*>(V + (int64_t)blockIdx.x * ld);
  U m = 0;
#pragma unroll 4
  for (int64_t i = threadIdx.x; i < rows; i += blockDim.x) {
    const U b = col[i] & kAbs;
    m = b > m ? b : m;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const U x = __shfl_xor_sync(0xffffffffu, m, o);
    m = x > m ? x : m;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : (U)0;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const U x = __shfl_xor_sync(0xffffffffu, m, o);
      m = x > m ? x : m;
    }
    if (threadIdx.x == 0) {
      if constexpr (sizeof(T) == 4) cexp[blockIdx.x] = exp_above(__uint_as_float(m));
      else cexp[blockIdx.x] = exp_above_d(__longlong_as_double((long long)m));
    }
  }
}

// S digits of an FP64 value, on the integer pipes (GB300's FP64 pipe runs ~2 operations per cycle
// and SM): r = x 2^(7 - e) (|r| <= 128) is rounded to the unit of the last digit, R = round(r
// 2^(8 (S - 1))) (nearest, ties to even), straight from x's bit pattern, and R is written in
// balanced base 256 from the lowest digit: a_s in [-128, 127] for s >= 1, |a_0| <= 128, and
// sum a_s 2^(-8 s) = R 2^(-8 (S - 1)); the digits come back as floats (exact).  Zeros and
// subnormal x give zero digits (a subnormal lies below 2^-1022, far under the last digit of any
// column whose largest entry is normal); a non-finite x, or one at or above 2^e (not possible for
// e from the column's maximum of finite entries), gives NaN digits, which the products carry on.
template <int S>
__device__ __forceinline__ void oz_digits_f64(double x, int e, float* af) {
  const long long bits = __double_as_longlong(x);
  const int E = (int)((bits >> 52) & 0x7ff);
  const int k = 1075 - E - 7 + e - 8 * (S - 1);                            // R = m 2^-k
  if (E == 0x7ff || (E != 0 && k < 1)) {
#pragma unroll
    for (int s = 0; s < S; ++s) af[s] = __int_as_float(0x7fc00000);
    return;
  }
  long long R = 0;
  if (E != 0) {
    const long long m = (bits & 0xfffffffffffffll) | 0x10000000000000ll;     // x = +-m 2^(E - 1075)
    if (k < 63) {
      R = m >> k;
      const long long rem = m & ((1ll << k) - 1), half = 1ll << (k - 1);
      if (rem > half || (rem == half && (R & 1))) ++R;
    }
    if (bits < 0) R = -R;
  }
#pragma unroll
  for (int s = S - 1; s >= 1; --s) {
    const int d = (int)((R + 128) & 255) - 128;
    af[s] = (float)d;
    R = (R - d) >> 8;                                                      // exact: R - d = 0 mod 256
  }
  af[0] = (float)R;
}

// Digit planes D[t] (cols x ld, the layout of V) of the column-scaled column-major V: for FP32 V
// by FP32 steps (each digit the rounded remainder, the next the remainder times 256, exact), for
// FP64 V on the integer pipes (oz_digits_f64).
template <typename T, int S>
__global__ void k_oz_split_cols(const T* __restrict__ V, int64_t ld, int64_t cols, const int* __restrict__ cexp,
                                __nv_bfloat16* __restrict__ D) {
  const int64_t total = ld * cols;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += st) {
    const int64_t j = idx / ld;
    const int e = cexp[j];
    float af[S];
    if constexpr (sizeof(T) == 4) {
      float r = ldexpf((float)V[idx], 7 - e);
#pragma unroll
      for (int s = 0; s < S; ++s) {
        af[s] = rintf(r);
        r = (r - af[s]) * 256.0f;                                         // exact
      }
    } else {
      oz_digits_f64<S>((double)V[idx], e, af);
    }
#pragma unroll
    for (int s = 0; s < S; ++s)   // an integer of magnitude <= 128 times 2^-8s: exact in BF16
      D[(int64_t)s * total + idx] = __float2bfloat16_rn(af[s] * __int_as_float((127 - 8 * s) << 23));
  }
}

// ---------------------------------------------------------------------------- Gramian operands
// For G = J^T diag(w) J: column maxima of |J| and of |w_n J_nj| over the points (row blocks of J
// in blockIdx.y, combined by atomicMax on the bit patterns of non-negative doubles, which order as
// the values do).  The second maximum is formed in FP32 with w rounded to FP32 and enlarged by
// 2^-20 of itself, an upper bound of the exact one.
__global__ void k_oz_gram_colmax(const float* __restrict__ J, int64_t ldJ, int64_t N, const double* __restrict__ w,
                                 int64_t rows_per, unsigned long long* __restrict__ mj,
                                 unsigned long long* __restrict__ mw) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ldJ) return;
  const int64_t n0 = (int64_t)blockIdx.y * rows_per, n1 = min(N, n0 + rows_per);
  float a = 0.f, b = 0.f;
  for (int64_t n = n0; n < n1; ++n) {
    const float x = fabsf(J[n * ldJ + j]);
    a = fmaxf(a, x);
    b = fmaxf(b, x * fabsf(f64_to_f32_rn(w[n])));
  }
  atomicMax(mj + j, (unsigned long long)__double_as_longlong((double)a));
  atomicMax(mw + j, (unsigned long long)__double_as_longlong((double)b * (1.0 + 0x1p-20)));
}

__global__ void k_oz_gram_exp(const unsigned long long* __restrict__ mj, const unsigned long long* __restrict__ mw,
                              int64_t n, int* __restrict__ ej, int* __restrict__ ew) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  ej[j] = exp_above_d(__longlong_as_double((long long)mj[j]));
  ew[j] = exp_above_d(__longlong_as_double((long long)mw[j]));
}

// Digit planes of the column-scaled J^T and (diag(w) J)^T, both p-major with the points
// contiguous (AT[s] and BT[s]: ldJ x ldN, columns n >= N zero), kDigG digits each: A from the FP32
// J (exact steps in FP32), B from the FP64 products w_n J_nj (digits on the integer pipes).
// 32 x 32 tiles, transposed through shared memory.
constexpr int kDigG = 6;

__global__ void k_oz_split_gram(const float* __restrict__ J, int64_t ldJ, int64_t N, const double* __restrict__ w,
                                const int* __restrict__ ej, const int* __restrict__ ew,
                                __nv_bfloat16* __restrict__ AT, __nv_bfloat16* __restrict__ BT, int64_t ldN) {
  __shared__ __nv_bfloat16 ta[kDigG][32][34], tb[kDigG][32][34];
  const int64_t j0 = (int64_t)blockIdx.x * 32, n0 = (int64_t)blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int64_t j = j0 + tx;
  const int ea = ej[j], eb = ew[j];
  for (int i = ty; i < 32; i += blockDim.y) {
    const int64_t n = n0 + i;
    float ra = 0.f;
    float b[kDigG];
    if (n < N) {
      const float x = J[n * ldJ + j];
      ra = x * __int_as_float((127 + 7 - ea) << 23);      // |ra| < 128, exact
      oz_digits_f64<kDigG>(w[n] * f32_to_f64(x), eb, b);  // |w_n J_nj 2^(7 - eb)| < 128
    } else {
#pragma unroll
      for (int s = 0; s < kDigG; ++s) b[s] = 0.f;
    }
#pragma unroll
    for (int s = 0; s < kDigG; ++s) {
      const float a = rintf(ra);
      ra = (ra - a) * 256.0f;                             // exact
      const float sc = __int_as_float((127 - 8 * s) << 23);
      ta[s][i][tx] = __float2bfloat16_rn(a * sc);         // integers of magnitude <= 128: exact
      tb[s][i][tx] = __float2bfloat16_rn(b[s] * sc);
    }
  }
  __syncthreads();
  for (int i = ty; i < 32; i += blockDim.y) {
    const int64_t jj = j0 + i, n = n0 + tx;
#pragma unroll
    for (int s = 0; s < kDigG; ++s) {
      AT[(int64_t)s * ldJ * ldN + jj * ldN + n] = ta[s][tx][i];
      BT[(int64_t)s * ldJ * ldN + jj * ldN + n] = tb[s][tx][i];
    }
  }
}

// ---------------------------------------------------------------------------- row-scaled FP64 operand
// For U = B W (B: p x ell column-major FP64, contracted over its columns): e_m of every row of B
// (max over the row's ell entries).  Block (32, 8): 32 rows (coalesced), eight column residues,
// the maximum taken on the magnitudes' bit patterns (non-negative doubles order as their bits) in
// the integer pipes.
__global__ void k_oz_rowexp_cm(const double* __restrict__ B, int64_t ldB, int64_t rows, int cols,
                               int* __restrict__ rexp) {
  __shared__ unsigned long long red[8][33];
  const int64_t m = (int64_t)blockIdx.x * 32 + threadIdx.x;
  unsigned long long mx = 0;
  if (m < rows) {
#pragma unroll 4
    for (int k = threadIdx.y; k < cols; k += 8) {
      const unsigned long long b = (unsigned long long)__double_as_longlong(B[m + (int64_t)k * ldB]) & 0x7fffffffffffffffull;
      mx = b > mx ? b : mx;
    }
  }
  red[threadIdx.y][threadIdx.x] = mx;
  __syncthreads();
  if (threadIdx.y == 0 && m < rows) {
#pragma unroll
    for (int y = 1; y < 8; ++y) mx = red[y][threadIdx.x] > mx ? red[y][threadIdx.x] : mx;
    rexp[m] = exp_above_d(__longlong_as_double((long long)mx));
  }
}

// Digit planes BT[s] (rows x ldK, K-major: row m's ell entries contiguous, k >= cols zero) of the
// row-scaled B, kDigZ digits per entry on the integer pipes; 32 x 32 tiles transposed through
// shared memory.
__global__ void k_oz_split_rows_cm(const double* __restrict__ B, int64_t ldB, int64_t rows, int cols,
                                   const int* __restrict__ rexp, __nv_bfloat16* __restrict__ BT, int64_t ldK) {
  __shared__ __nv_bfloat16 tile[kDigZ][32][34];
  const int64_t m0 = (int64_t)blockIdx.x * 32;
  const int k0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int i = ty; i < 32; i += blockDim.y) {            // column k0 + i, rows m0 + tx (coalesced)
    const int64_t m = m0 + tx;
    const int k = k0 + i;
    float a[kDigZ];
    if (m < rows && k < cols) {
      oz_digits_f64<kDigZ>(B[m + (int64_t)k * ldB], rexp[m], a);
    } else {
#pragma unroll
      for (int q = 0; q < kDigZ; ++q) a[q] = 0.f;
    }
#pragma unroll
    for (int q = 0; q < kDigZ; ++q)
      tile[q][tx][i] = __float2bfloat16_rn(a[q] * __int_as_float((127 - 8 * q) << 23));
  }
  __syncthreads();
  for (int i = ty; i < 32; i += blockDim.y) {            // row m0 + i, entries k0 + tx (coalesced)
    const int64_t m = m0 + i;
    if (m >= rows) continue;
#pragma unroll
    for (int q = 0; q < kDigZ; ++q) BT[(int64_t)q * rows * ldK + m * ldK + k0 + tx] = tile[q][i][tx];
  }
}

// Ws (cols x ldK, column j at Ws + j ldK) = W[:, j] * colscale[j] (W: rows x cols column-major,
// leading dimension ldW), rows rows..ldK-1 zero.
__global__ void k_oz_scale_pad(const double* __restrict__ W, int64_t ldW, int rows, int cols,
                               const double* __restrict__ colscale, double* __restrict__ Ws, int64_t ldK) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)cols * ldK) return;
  const int64_t j = idx / ldK, k = idx - j * ldK;
  Ws[idx] = k < rows ? W[k + j * ldW] * colscale[j] : 0.0;
}

// ---------------------------------------------------------------------------- digit-plane GEMM
// (a.hi + a.lo) + b for an FP32 b, renormalised (df_add with b's low word zero, one add fewer)
__device__ __forceinline__ DF df_add_f(DF a, float b) {
  float s, e;
  two_sum(a.hi, b, s, e);
  e += a.lo;
  const float hi = s + e;
  return DF{hi, e - (hi - s)};
}

// Accumulator of the level s + t: levels 0..3 exact, levels 4.. shared (TMEM columns acc * kBN).
__host__ __device__ constexpr int acc_of(int level) { return level < 4 ? level : 4; }

// Shared-memory plan of the digit-plane GEMM: a ring of RB = 2 SB B-tile slots (two k-blocks of B
// digit tiles) and a ring of RA A-tile slots, as many as fit (at most 8).  When one k-block of A
// tiles does not fit beside two of B (SA = SB = 6), A gets one k-block and B every slot left
// (RB >= SB): the MMA issuer frees B tiles highest digit first, the order in which the producer
// refills them, so the next k-block's B tiles land in slots freed before the current one ends.
template <int SA, int SB>
struct OzSmem {
  static constexpr int kLimit = 232448;                                    // 227 KB per block
  static constexpr int kFixed = 1024 + 1024;                               // alignment, barriers
  static constexpr int kAvail = kLimit - kFixed;
  static constexpr bool kTwoB = kAvail - 2 * SB * kTileB >= SA * kTile;
  static constexpr int RB0 = (kAvail - SA * kTile) / kTileB;
  static constexpr int RB = kTwoB ? 2 * SB : (RB0 > 2 * SB ? 2 * SB : RB0);
  static constexpr int RA0 = (kAvail - RB * kTileB) / kTile;
  static constexpr int RA = RA0 > 8 ? 8 : RA0;
  static constexpr int bytes = RA * kTile + RB * kTileB + kFixed;
};

constexpr int kEpiWarps = 16;                      // four warps per TMEM lane quarter
constexpr int kOzThreads = 32 * (2 + kEpiWarps);
constexpr int kEpiT = kEpiWarps * 32;              // epilogue threads
constexpr int kColW = kBN / (kEpiWarps / 4);       // accumulator columns each epilogue thread drains
constexpr int kEpiG = 8;                           // columns per tcgen05.ld

// Work items of the digit-plane GEMM: output tiles of kBM x kBN (all of them, or for a symmetric
// product only the tiles that hold an entry on or below the diagonal, m >= n) times K slices of
// cps chunks, item = tile + tiles * slice.  Tiles are enumerated M-tile-major with the N tile
// fastest, so that consecutive items (taken by neighbouring CTAs) share their A digit tiles.
struct OzItems {
  int n_tiles, m_tiles, tiles;   // tiles: number of enumerated tiles
  int lower;                     // enumerate only tiles with an entry m >= n
  int nks, cps;                  // K slices of this launch; chunks per slice
  int chunk0, chunk_end;         // chunks [chunk0, chunk_end) of this launch
};

// Tiles of M-tile row mt that hold an entry m >= n.
__host__ __device__ __forceinline__ int oz_lower_count(int mt, int n_tiles) {
  const int c = ((mt + 1) * kBM - 1) / kBN + 1;
  return c < n_tiles ? c : n_tiles;
}

__device__ __forceinline__ void oz_item(const OzItems& it, int item, int& mt, int& nt, int& ks, int& c_lo,
                                        int& c_hi) {
  int tile = item % it.tiles;
  ks = item / it.tiles;
  if (!it.lower) {
    nt = tile % it.n_tiles;
    mt = tile / it.n_tiles;
  } else {
    // item < tiles * nks, so the walk ends within the m_tiles rows
    mt = 0;
    for (int cnt = oz_lower_count(0, it.n_tiles); tile >= cnt; cnt = oz_lower_count(mt, it.n_tiles)) {
      tile -= cnt;
      ++mt;
    }
    nt = tile;
  }
  c_lo = it.chunk0 + ks * it.cps;
  c_hi = c_lo + it.cps < it.chunk_end ? c_lo + it.cps : it.chunk_end;
}

// Final scaled output written by the epilogue itself (one K slice covering all of K):
// out[n * ldOut + m] = 2^(rexp[m] + cexp[n] - 14) v for m < M, n < Nout (and m >= n when lower).
struct OzDirect {
  const int* rexp;
  const int* cexp;
  double* out;
  int64_t ldOut, M, Nout;
  int on;
  int sub;                          // subtract from out instead of writing it
};

// x 2^E for a double x built from an FP32 value (normal range), by integer exponent arithmetic
// (GB300's FP64 pipe is narrow); ldexp where the result would leave the normal range.
__device__ __forceinline__ double oz_scale(double x, int E) {
  if (x == 0.0) return 0.0;
  const long long b = __double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7ff) + E;
  if (ex < 1 || ex > 2046) return ldexp(x, E);
  return __longlong_as_double(b + ((long long)E << 52));
}

// D = sum over kept (s, t) of A_s B_t^T.  A planes (tmA: cols = K, rows = M, planes = SA), B
// planes (tmB: cols = K, rows = Nout, planes = SB), both K-major.  The persistent CTAs take items
// blockIdx.x, blockIdx.x + gridDim.x, ...; an item runs the chunks of its K slice one after the
// other through the TMEM accumulators, and the epilogue adds each chunk's double-float value to a
// running sum (run: per CTA and epilogue thread, 48 float2, L2-resident) in chunk order.  At the
// slice's last chunk the epilogue writes the slice's partial (hi, lo) of output (m, n) at
// P[(slice * ldL + n) * ldM + m], or with d.on the scaled float64 output itself.  While the
// epilogue warps drain one chunk's accumulators, the producer already loads the next chunk's
// tiles; the MMA issuer waits for the drain (accumulator-empty barrier) before it writes the
// accumulators again.
template <int SA, int SB>
__global__ void __launch_bounds__(kOzThreads, 1) k_oz_gemm(const __grid_constant__ CUtensorMap tmA,
                                                          const __grid_constant__ CUtensorMap tmB, int64_t K,
                                                          const OzItems it, float2* __restrict__ P, int64_t ldL,
                                                          int64_t ldM, float2* __restrict__ run, const OzDirect d,
                                                          int* status, long long wait_cycles) {
  static_assert(SB - 1 <= kLevels && SA - 1 <= kLevels, "every digit plane takes part in a kept pair");
  using SP = OzSmem<SA, SB>;
  constexpr int RA = SP::RA, RB = SP::RB;
  // a k-block's tiles fit the rings together: a tile only waits for a slot of an earlier k-block,
  // which the MMA issuer can always finish (no circular wait)
  static_assert(RA >= SA && RB >= SB, "one k-block of digit tiles must fit the rings");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* ringA = smem;
  uint8_t* ringB = smem + RA * kTile;
  uint64_t* fullA = reinterpret_cast<uint64_t*>(ringB + RB * kTileB);
  uint64_t* emptyA = fullA + RA;
  uint64_t* fullB = emptyA + RA;
  uint64_t* emptyB = fullB + RB;
  uint64_t* acc_full = emptyB + RB;
  uint64_t* acc_empty = acc_full + 1;
  uint64_t* mma_done = acc_empty + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int items = it.tiles * it.nks;

  if (threadIdx.x == 0) {
    for (int i = 0; i < RA; ++i) {
      mbar_init(&fullA[i], 1);
      mbar_init(&emptyA[i], 1);
    }
    for (int i = 0; i < RB; ++i) {
      mbar_init(&fullB[i], 1);
      mbar_init(&emptyB[i], 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, kEpiWarps);
    mbar_init(mma_done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tmem_slot, 512);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  int err = 0;

  if (warp == 0 && lane == 0) {
    // ---------------------------------------------------------------- TMA producer
    int iA = 0, iB = 0;
    for (int item = blockIdx.x; item < items && !*abort_flag; item += gridDim.x) {
      int mt, nt, ks, c_lo, c_hi;
      oz_item(it, item, mt, nt, ks, c_lo, c_hi);
      // the k-blocks of the slice's chunks (every chunk but the last of K is kChunk long)
      const int64_t k_end = (int64_t)c_hi * kChunk < K ? (int64_t)c_hi * kChunk : K;
      for (int64_t x0 = (int64_t)c_lo * kChunk; x0 < k_end && !*abort_flag; x0 += kBK) {
        const int x = (int)x0;
        for (int q = 0; q < SA + SB; ++q) {
          const bool isB = q < SB;
          const int i = isB ? iB : iA, R = isB ? RB : RA;
          uint64_t* fb = isB ? &fullB[i % R] : &fullA[i % R];
          uint64_t* eb = isB ? &emptyB[i % R] : &emptyA[i % R];
          if (i >= R && !mbar_wait(eb, ((i / R) - 1) & 1, wait_cycles)) {
            err |= 1;
            *abort_flag = 1;
            break;
          }
          if (isB) {
            mbar_expect_tx(fb, kTileB);
            tma_load_3d(ringB + (i % RB) * kTileB, &tmB, x, nt * kBN, SB - 1 - q, fb);
            ++iB;
          } else {
            mbar_expect_tx(fb, kTile);
            tma_load_3d(ringA + (i % RA) * kTile, &tmA, x, mt * kBM, q - SB, fb);
            ++iA;
          }
        }
      }
    }
    // every load still unconsumed must land before the CTA may exit
    for (int j = iA > RA ? iA - RA : 0; j < iA; ++j)
      if (!mbar_wait(&fullA[j % RA], (j / RA) & 1, kDrainCycles)) err |= 2;
    for (int j = iB > RB ? iB - RB : 0; j < iB; ++j)
      if (!mbar_wait(&fullB[j % RB], (j / RB) & 1, kDrainCycles)) err |= 2;
  } else if (warp == 1 && lane == 0) {
    // ---------------------------------------------------------------- MMA issuer
    constexpr uint32_t idesc = make_idesc(1u, kBM, kBN);
    int iA = 0, iB = 0, nsub = 0;        // nsub: chunks run through the accumulators so far
    bool ok = true, pending = false;   // pending: MMAs of the current chunk not yet committed
    for (int item = blockIdx.x; item < items && ok; item += gridDim.x) {
      int mt, nt, ks, c_lo, c_hi;
      oz_item(it, item, mt, nt, ks, c_lo, c_hi);
      for (int c = c_lo; c < c_hi && ok; ++c, ++nsub) {
        const int64_t k0 = (int64_t)c * kChunk;
        const int nkb = (int)(((K - k0 < kChunk ? K - k0 : kChunk) + kBK - 1) / kBK);
        // the epilogue has read the previous chunk's accumulators
        if (nsub > 0 && (*abort_flag || !mbar_wait(acc_empty, (nsub - 1) & 1, wait_cycles))) {
          ok = false;
          break;
        }
        fence_after();
        uint32_t started = 0;
        for (int kb = 0; kb < nkb && ok; ++kb) {
          if (*abort_flag) {
            ok = false;
            break;
          }
          // The k-block's tiles sit at counters iB .. iB + SB - 1 (B, digit SB - 1 - q at iB + q) and
          // iA .. iA + SA - 1 (A, digit s at iA + s); their ring slots wrap at most once.  The MMAs
          // are issued in straight-line code (digit loops unrolled, slots computed once): a branch
          // between tcgen05.mma instructions measured ~90 cycles each on GB300, an MMA ~56.
          const int sb0 = iB % RB, sa0 = iA % RA;
          const uint32_t pb0 = (uint32_t)(iB / RB) & 1u, pa0 = (uint32_t)(iA / RA) & 1u;
          uint64_t bdesc[SB];
          int bslot[SB];
#pragma unroll
          for (int q = 0; q < SB; ++q) {
            const bool wrap = sb0 + q >= RB;
            const int sl = wrap ? sb0 + q - RB : sb0 + q;
            if (ok && !mbar_wait(&fullB[sl], wrap ? pb0 ^ 1u : pb0, wait_cycles)) ok = false;
            bdesc[SB - 1 - q] = make_desc(ringB + sl * kTileB);
            bslot[SB - 1 - q] = sl;
          }
          if (!ok) break;
#pragma unroll
          for (int s = 0; s < SA; ++s) {
            const bool wrap = sa0 + s >= RA;
            const int sl = wrap ? sa0 + s - RA : sa0 + s;
            if (!mbar_wait(&fullA[sl], wrap ? pa0 ^ 1u : pa0, wait_cycles)) {
              ok = false;
              break;
            }
            fence_after();
            const uint64_t ad = make_desc(ringA + sl * kTile);
#pragma unroll
            for (int t = 0; t < SB; ++t) {
              if (s + t > kLevels) continue;
              const int acc = acc_of(s + t);
              const uint32_t accf = (started >> acc) & 1u;
#pragma unroll
              for (int k = 0; k < kBK / 16; ++k)
                mma_bf16(tmem + (uint32_t)(acc * kBN), ad + (uint64_t)(k * 2), bdesc[t] + (uint64_t)(k * 2), idesc,
                         accf | (uint32_t)(k > 0));
              started |= 1u << acc;
              pending = true;
            }
            mma_commit(&emptyA[sl]);                                    // A_s is done
#pragma unroll
            for (int t = 0; t < SB; ++t)                                // B_t after its last pair
              if ((SA - 1 < kLevels - t ? SA - 1 : kLevels - t) == s) mma_commit(&emptyB[bslot[t]]);
          }
          iA += SA;
          iB += SB;
        }
        if (!ok) break;
        mma_commit(acc_full);          // arrives once this chunk's MMAs have completed
        pending = false;
      }
    }
    if (!ok) {
      err |= 1;
      *abort_flag = 1;
      if (pending) mma_commit(acc_full);   // the phase an epilogue warp may be waiting on
    }
    // every MMA this thread issued has completed before the tensor memory is freed
    mma_commit(mma_done);
    if (!mbar_wait(mma_done, 0, kDrainCycles)) err |= 2;
  } else if (warp >= 2) {
    // ---------------------------------------------------------------- epilogue
    const int ew = warp - 2;
    const int q = warp & 3;                       // TMEM lane quarter this warp may access
    const int part = ew >> 2;                     // which kColW-wide part of the kBN columns
    const uint32_t lane_addr = tmem + ((uint32_t)(q * 32) << 16);
    // accumulators some kept pair writes (the MMA issuer's first write to each clears it)
    uint32_t started = 0;
#pragma unroll
    for (int s = 0; s < SA; ++s)
#pragma unroll
      for (int t = 0; t < SB; ++t)
        if (s + t <= kLevels) started |= 1u << acc_of(s + t);
    // running sums of this thread's kColW outputs: element e at my_run[e * kEpiT] (coalesced per warp)
    float2* my_run = run ? run + (int64_t)blockIdx.x * (kEpiT * kColW) + (ew * 32 + lane) : nullptr;
    int nsub = 0;
    bool stop = false;
    for (int item = blockIdx.x; item < items && !stop; item += gridDim.x) {
      int mt, nt, ks, c_lo, c_hi;
      oz_item(it, item, mt, nt, ks, c_lo, c_hi);
      const int64_t row = (int64_t)mt * kBM + q * 32 + lane;
      for (int c = c_lo; c < c_hi; ++c, ++nsub) {
        // wait for the chunk's accumulators; give up when another role aborted (the MMA issuer
        // then waits for its own MMAs before the tensor memory is freed)
        int got = 0;
        if (lane == 0) {
          const long long t0 = clock64();
          while (true) {
            if (mbar_try_wait(acc_full, nsub & 1)) { got = 1; break; }
            if (*abort_flag) break;
            if (clock64() - t0 > wait_cycles) {
              err |= 1;
              *abort_flag = 1;
              break;
            }
          }
        }
        got = __shfl_sync(0xffffffffu, got, 0);
        __syncwarp();
        fence_after();
        if (!got || *abort_flag) {
          stop = true;
          break;
        }
        const bool first = c == c_lo, last = c + 1 == c_hi;
        for (int c0 = part * kColW; c0 < (part + 1) * kColW; c0 += kEpiG) {
          uint32_t e[kAcc][kEpiG];
#pragma unroll
          for (int a = 0; a < kAcc; ++a) tmem_ld8(lane_addr + (uint32_t)(a * kBN + c0), e[a]);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < kEpiG; ++j) {
            // exact parts: E0 integer, E1..E3 in 2^-8, 2^-16, 2^-24 units, each within 2^24 units;
            // added from the smallest: the pair keeps ~48 bits of their sum, then the rounded
            // levels 4..
            DF v{0.0f, 0.0f};
            bool init = false;                                  // resolved at compile time
#pragma unroll
            for (int a = kAcc - 1; a >= 0; --a)
              if (started & (1u << a)) {
                const float x = __uint_as_float(e[a][j]);
                if (!init) v = DF{x, 0.0f};
                else v = df_add_f(v, x);
                init = true;
              }
            float2* rp = my_run + (int64_t)(c0 - part * kColW + j) * kEpiT;
            if (!first) {
              const float2 r = *rp;
              v = df_add(DF{r.x, r.y}, v);
            }
            if (!last) {
              *rp = make_float2(v.hi, v.lo);
              continue;
            }
            const int64_t n = (int64_t)nt * kBN + c0 + j;
            if (!d.on) {
              P[((int64_t)ks * ldL + n) * ldM + row] = make_float2(v.hi, v.lo);
            } else if (row < d.M && n < d.Nout && (!it.lower || row >= n)) {
              double* o = d.out + n * d.ldOut + row;
              const double val = oz_scale(f32_to_f64(v.hi) + f32_to_f64(v.lo), d.rexp[row] + d.cexp[n] - 14);
              *o = d.sub ? *o - val : val;
            }
          }
        }
        fence_before();
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(acc_empty)) : "memory");
      }
    }
  }
  __syncwarp();
  if (err && status) atomicOr(status, (err & 2) ? (kStatTimeout | kStatDrain) : kStatTimeout);
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// Sum of the partials of chunks [0, nc) of output (m, j) in chunk order (double-float), added to
// the running sum acc when !first, stored back to acc when !last; when last, scaled and written as
// float64: MODE 1 (Z'' = diag(w) diag(2^e) J Omega): out[j * ldOut + m] = w_m 2^(2 e_m + f_j - 14)
// v; MODE 2 (Y): out[j * ldOut + m] = 2^(f_j - 14) v; MODE 3 (a product of a row-scaled and a
// column-scaled operand): out[j * ldOut + m] = 2^(e_m + f_j - 14) v.  Rows M <= m < ldOut are
// written as zero.  With lower, entries m < j (whose partials a lower-tile GEMM may not have
// written) are left untouched.
template <int MODE>
__global__ void k_oz_reduce(const float2* __restrict__ P, int nc, int64_t ldL, int64_t ldM, float2* __restrict__ acc,
                            int first, int last, int64_t M, int64_t ldOut, const int* __restrict__ rexp,
                            const int* __restrict__ cexp, const double* __restrict__ w, double* __restrict__ out,
                            int lower) {
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t j = blockIdx.y;
  if (m >= ldOut) return;
  if (m >= M) {
    if (last) out[j * ldOut + m] = 0.0;
    return;
  }
  if (lower && m < j) return;
  DF v{0.0f, 0.0f};
  if (!first) {
    const float2 a = acc[j * ldM + m];
    v = DF{a.x, a.y};
  }
  for (int c = 0; c < nc; ++c) {
    const float2 x = P[((int64_t)c * ldL + j) * ldM + m];
    v = df_add(v, DF{x.x, x.y});
  }
  if (!last) {
    acc[j * ldM + m] = make_float2(v.hi, v.lo);
    return;
  }
  const double x = f32_to_f64(v.hi) + f32_to_f64(v.lo);
  if (MODE == 1)
    out[j * ldOut + m] = w[m] * ldexp(x, 2 * rexp[m] + cexp[j] - 14);
  else if (MODE == 2)
    out[j * ldOut + m] = ldexp(x, cexp[j] - 14);
  else
    out[j * ldOut + m] = ldexp(x, rexp[m] + cexp[j] - 14);
}

}  // namespace

// ---------------------------------------------------------------------------- host
struct OzSketch {
  __nv_bfloat16 *JD = nullptr, *JDT = nullptr, *OD = nullptr, *ZD = nullptr;
  size_t JD_b = 0, JDT_b = 0, OD_b = 0, ZD_b = 0;
  int *jexp = nullptr, *oexp = nullptr, *zexp = nullptr;
  size_t jexp_b = 0, oexp_b = 0, zexp_b = 0;
  double* Zs = nullptr;   size_t Zs_b = 0;     // Z'' transposed: ell x ldN
  // the Gramian's operands (column-scaled J^T and (diag(w) J)^T digit planes) and exponents
  __nv_bfloat16 *GA = nullptr, *GB = nullptr;
  size_t GA_b = 0, GB_b = 0;
  int* gexp = nullptr;    size_t gexp_b = 0;   // 2 ldJ: exponents of J's and of diag(w) J's columns
  unsigned long long* gmax = nullptr; size_t gmax_b = 0;
  float2* part = nullptr; size_t part_b = 0;   // split-K partials of one launch
  float2* acc = nullptr;  size_t acc_b = 0;    // running sums across launches
  float2* run = nullptr;  size_t run_b = 0;    // per-CTA running sums of the chunks of a K slice
  // the factor's Gram products: digit planes of an FP64 p x ell operand and its column exponents
  __nv_bfloat16* FD = nullptr; size_t FD_b = 0;
  int* fexp = nullptr;    size_t fexp_b = 0;
  // U = B W: digit planes of the row-scaled B (K-major) and of the column-scaled W, exponents
  __nv_bfloat16 *UA = nullptr, *UB = nullptr;
  size_t UA_b = 0, UB_b = 0;
  int *uexp = nullptr, *wexp = nullptr;
  size_t uexp_b = 0, wexp_b = 0;
  double* Ws = nullptr;   size_t Ws_b = 0;
  // the Jacobian the digit planes were made from
  const float* J = nullptr;
  int64_t N = 0, ldJ = 0, ldN = 0;
  uint64_t j_version = ~0ull;
};

namespace {

template <typename P>
cudaError_t grow(P** p, size_t* cap, size_t bytes) {
  if (bytes <= *cap) return cudaSuccess;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e == cudaSuccess) *cap = bytes;
  return e;
}

// Tiles a lower-triangle digit-plane GEMM enumerates.
int64_t oz_lower_tiles(int m_tiles, int n_tiles) {
  int64_t t = 0;
  for (int m = 0; m < m_tiles; ++m) t += oz_lower_count(m, n_tiles);
  return t;
}

// D[m, n] = sum over kept digit pairs for an M x Nout output and K columns, into out (float64,
// MODE as k_oz_reduce; with lower only the entries m >= n, of tiles that hold one).  K is cut into
// slices of up to max_cps chunks of kChunk, as few as keep four items per SM; each item sums its
// slice's chunks in order.  With MODE 3 and one slice the GEMM's epilogue writes out itself;
// otherwise the slices' partials go to launches of at most partial_cap bytes, each followed by the
// fixed-order reduction, their sums carried in the running double-float sums.
template <int SA, int SB, int MODE>
cudaError_t run_digit_gemm(OzSketch* o, const CUtensorMap& tmA, const CUtensorMap& tmB, int64_t M, int64_t Nout,
                           int64_t K, const int* rexp, const int* cexp, const double* w, double* out, int64_t ldOut,
                           int* status, cudaStream_t s, long long wait_cycles, bool lower = false, int max_cps = 1,
                           size_t partial_cap = kPartialCap, bool sub = false) {
  const int64_t ldL = rup(Nout, kBN), ldM = rup(M, kBM);
  const int64_t nchunks = (K + kChunk - 1) / kChunk;
  const size_t chunk_bytes = (size_t)ldL * ldM * sizeof(float2);
  auto kern = k_oz_gemm<SA, SB>;
  constexpr int smem = OzSmem<SA, SB>::bytes;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess) return e;
  int dev = 0, nsm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int n_tiles = (int)(ldL / kBN), m_tiles = (int)(ldM / kBM);
  const int64_t tiles = lower ? oz_lower_tiles(m_tiles, n_tiles) : (int64_t)n_tiles * m_tiles;
  int64_t nks = std::min<int64_t>(nchunks, std::max<int64_t>(1, (4 * (int64_t)nsm + tiles - 1) / tiles));
  const int64_t cps = std::min<int64_t>(std::max(1, max_cps), (nchunks + nks - 1) / nks);
  nks = (nchunks + cps - 1) / cps;
  if (cps > 1) {
    const size_t run_bytes = (size_t)std::min<int64_t>(tiles * nks, nsm) * kEpiT * kColW * sizeof(float2);
    if ((e = grow(&o->run, &o->run_b, run_bytes)) != cudaSuccess) return e;
  }
  OzDirect d{rexp, cexp, out, ldOut, M, Nout, 0, sub ? 1 : 0};
  if (sub && !(MODE == 3 && nks == 1)) return cudaErrorInvalidValue;   // subtraction: one slice only
  if (MODE == 3 && nks == 1) {
    d.on = 1;
    const OzItems it{n_tiles, m_tiles, (int)tiles, lower ? 1 : 0, 1, (int)cps, 0, (int)nchunks};
    const unsigned grid = (unsigned)std::min<int64_t>(tiles, nsm);
    kern<<<grid, kOzThreads, smem, s>>>(tmA, tmB, K, it, nullptr, ldL, ldM, o->run, d, status, wait_cycles);
    note_launch();
    return cudaGetLastError();
  }
  const int64_t slice_bytes = (int64_t)chunk_bytes;
  const int64_t per_launch = std::max<int64_t>(1, std::min<int64_t>(nks, (int64_t)(partial_cap / slice_bytes)));
  if ((e = grow(&o->part, &o->part_b, chunk_bytes * per_launch)) != cudaSuccess) return e;
  if (per_launch < nks && (e = grow(&o->acc, &o->acc_b, chunk_bytes)) != cudaSuccess) return e;
  for (int64_t s0 = 0; s0 < nks; s0 += per_launch) {
    const int ns = (int)std::min<int64_t>(per_launch, nks - s0);
    const OzItems it{n_tiles, m_tiles, (int)tiles, lower ? 1 : 0, ns, (int)cps, (int)(s0 * cps),
                     (int)std::min<int64_t>(nchunks, (s0 + ns) * cps)};
    const unsigned grid = (unsigned)std::min<int64_t>(tiles * ns, nsm);
    kern<<<grid, kOzThreads, smem, s>>>(tmA, tmB, K, it, o->part, ldL, ldM, o->run, d, status, wait_cycles);
    note_launch();
    dim3 rg((unsigned)((ldOut + 255) / 256), (unsigned)Nout);
    k_oz_reduce<MODE><<<rg, 256, 0, s>>>(o->part, ns, ldL, ldM, o->acc, s0 == 0, s0 + ns >= nks, M, ldOut, rexp,
                                         cexp, w, out, lower ? 1 : 0);
    note_launch();
  }
  return cudaGetLastError();
}

}  // namespace

OzSketch* oz_create() { return new (std::nothrow) OzSketch(); }

void oz_destroy(OzSketch* o) {
  if (!o) return;
  void* bufs[] = {o->JD, o->JDT, o->OD, o->ZD, o->jexp, o->oexp, o->zexp, o->Zs, o->part, o->acc,
                  o->GA, o->GB, o->gexp, o->gmax, o->run, o->FD, o->fexp, o->UA, o->UB, o->uexp, o->wexp,
                  o->Ws};
  for (void* b : bufs)
    if (b) cudaFree(b);
  delete o;
}

cudaError_t oz_sketch(OzSketch* o, const float* J, int64_t ldJ, int64_t N, int64_t p, uint64_t j_version,
                      const float* Omega, int64_t ldY, int ell, const double* w, double* Y64, const char** why,
                      cudaStream_t s, int* status, long long wait_cycles) {
  *why = nullptr;
  if (!tensor_map_encoder()) {
    *why = "cuTensorMapEncodeTiled unavailable";
    return cudaSuccess;
  }
  if ((ldJ % 32) || (ldY % 32) || ldY != ldJ || N < 1 || ell < 1) {
    *why = "leading dimensions must be equal multiples of 32";
    return cudaSuccess;
  }
  const int64_t ldN = rup(N, 32);
  cudaError_t e;
  // digit planes of J, once per Jacobian
  if (o->J != J || o->j_version != j_version || o->N != N || o->ldJ != ldJ) {
    if ((e = grow(&o->JD, &o->JD_b, (size_t)kDigJ * N * ldJ * 2)) != cudaSuccess) return e;
    if ((e = grow(&o->JDT, &o->JDT_b, (size_t)kDigJ * ldJ * ldN * 2)) != cudaSuccess) return e;
    if ((e = grow(&o->jexp, &o->jexp_b, (size_t)N * sizeof(int))) != cudaSuccess) return e;
    k_oz_rowexp<<<(unsigned)((N + 7) / 8), 256, 0, s>>>(J, ldJ, N, o->jexp);
    note_launch();
    dim3 blk(32, 8), grd((unsigned)(ldJ / 32), (unsigned)(ldN / 32));
    k_oz_split_rows<<<grd, blk, 0, s>>>(J, ldJ, N, o->jexp, o->JD, o->JDT, ldN);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    o->J = J;
    o->j_version = j_version;
    o->N = N;
    o->ldJ = ldJ;
    o->ldN = ldN;
  }
  // digit planes of Omega
  if ((e = grow(&o->OD, &o->OD_b, (size_t)kDigOm * ell * ldY * 2)) != cudaSuccess) return e;
  if ((e = grow(&o->oexp, &o->oexp_b, (size_t)ell * sizeof(int))) != cudaSuccess) return e;
  if ((e = grow(&o->zexp, &o->zexp_b, (size_t)ell * sizeof(int))) != cudaSuccess) return e;
  if ((e = grow(&o->Zs, &o->Zs_b, (size_t)ell * ldN * sizeof(double))) != cudaSuccess) return e;
  if ((e = grow(&o->ZD, &o->ZD_b, (size_t)kDigZ * ell * ldN * 2)) != cudaSuccess) return e;
  k_oz_colexp<float><<<(unsigned)ell, 256, 0, s>>>(Omega, ldY, p, o->oexp);
  note_launch();
  {
    const int64_t tot = ldY * ell;
    k_oz_split_cols<float, kDigOm><<<(unsigned)std::min<int64_t>((tot + 255) / 256, 8192), 256, 0, s>>>(
        Omega, ldY, ell, o->oexp, o->OD);
    note_launch();
  }
  CUtensorMap mA1, mB1, mA2, mB2;
  if (!make_tile_map(&mA1, o->JD, 2, N, ldJ, ldJ, kDigJ, N * ldJ, kBM) ||
      !make_tile_map(&mB1, o->OD, 2, ell, ldY, ldY, kDigOm, (int64_t)ell * ldY, kBN) ||
      !make_tile_map(&mA2, o->JDT, 2, ldJ, ldN, ldN, kDigJ, ldJ * ldN, kBM) ||
      !make_tile_map(&mB2, o->ZD, 2, ell, ldN, ldN, kDigZ, (int64_t)ell * ldN, kBN)) {
    *why = "tensor map encoding failed";
    return cudaSuccess;
  }
  // GEMM1: Z'' (ell x ldN, transposed) = diag(w) diag(2^e) J Omega
  if ((e = run_digit_gemm<kDigJ, kDigOm, 1>(o, mA1, mB1, N, ell, ldJ, o->jexp, o->oexp, w, o->Zs, ldN, status, s,
                                            wait_cycles)) != cudaSuccess)
    return e;
  k_oz_colexp<double><<<(unsigned)ell, 256, 0, s>>>(o->Zs, ldN, N, o->zexp);
  note_launch();
  {
    const int64_t tot = ldN * ell;
    k_oz_split_cols<double, kDigZ><<<(unsigned)std::min<int64_t>((tot + 255) / 256, 8192), 256, 0, s>>>(
        o->Zs, ldN, ell, o->zexp, o->ZD);
    note_launch();
  }
  // GEMM2: Y = J^T Z''
  return run_digit_gemm<kDigJ, kDigZ, 2>(o, mA2, mB2, p, ell, ldN, nullptr, o->zexp, nullptr, Y64, ldY, status, s,
                                         wait_cycles);
}

cudaError_t oz_gram(OzSketch* o, const float* J, int64_t ldJ, int64_t N, int64_t p, const double* w, double* G,
                    int64_t ldG, const char** why, cudaStream_t s, int* status, long long wait_cycles) {
  *why = nullptr;
  if (!tensor_map_encoder()) {
    *why = "cuTensorMapEncodeTiled unavailable";
    return cudaSuccess;
  }
  if ((ldJ % 32) || N < 1 || p < 1 || ldG < p) {
    *why = "the Jacobian's leading dimension must be a multiple of 32";
    return cudaSuccess;
  }
  const int64_t ldN = rup(N, 32);
  cudaError_t e;
  if ((e = grow(&o->GA, &o->GA_b, (size_t)kDigG * ldJ * ldN * 2)) != cudaSuccess) return e;
  if ((e = grow(&o->GB, &o->GB_b, (size_t)kDigG * ldJ * ldN * 2)) != cudaSuccess) return e;
  if ((e = grow(&o->gexp, &o->gexp_b, (size_t)2 * ldJ * sizeof(int))) != cudaSuccess) return e;
  if ((e = grow(&o->gmax, &o->gmax_b, (size_t)2 * ldJ * sizeof(unsigned long long))) != cudaSuccess) return e;
  int* ej = o->gexp;
  int* ew = o->gexp + ldJ;
  if ((e = cudaMemsetAsync(o->gmax, 0, (size_t)2 * ldJ * sizeof(unsigned long long), s)) != cudaSuccess) return e;
  {
    const int64_t rows_per = 256;
    dim3 g((unsigned)((ldJ + 255) / 256), (unsigned)((N + rows_per - 1) / rows_per));
    k_oz_gram_colmax<<<g, 256, 0, s>>>(J, ldJ, N, w, rows_per, o->gmax, o->gmax + ldJ);
    note_launch();
    k_oz_gram_exp<<<(unsigned)((ldJ + 255) / 256), 256, 0, s>>>(o->gmax, o->gmax + ldJ, ldJ, ej, ew);
    note_launch();
    dim3 blk(32, 8), grd((unsigned)(ldJ / 32), (unsigned)(ldN / 32));
    k_oz_split_gram<<<grd, blk, 0, s>>>(J, ldJ, N, w, ej, ew, o->GA, o->GB, ldN);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  CUtensorMap mA, mB;
  if (!make_tile_map(&mA, o->GA, 2, ldJ, ldN, ldN, kDigG, ldJ * ldN, kBM) ||
      !make_tile_map(&mB, o->GB, 2, ldJ, ldN, ldN, kDigG, ldJ * ldN, kBN)) {
    *why = "tensor map encoding failed";
    return cudaSuccess;
  }
  // G[j', j] = 2^(e_j' + f_j - 14) sum over kept pairs of AT_s BT_t^T for j' >= j, on the tiles of
  // the lower triangle.  Up to 16 K chunks: each tile summed over all of K by one CTA and written by
  // the GEMM's epilogue.  Longer K: one-chunk slices whose partials (up to 8 GB per launch) the
  // reduction adds, which measured faster than the CTA's running sums (3-D Poisson, p = 8641,
  // 43 chunks: 186 ms per NGD full step against 194, the same G bit for bit).
  const int64_t nchunks = (ldN + 255) / 256;
  return run_digit_gemm<kDigG, kDigG, 3>(o, mA, mB, p, p, ldN, ej, ew, nullptr, G, ldG, status, s, wait_cycles,
                                         true, nchunks <= 16 ? 1 << 30 : 1, size_t(8) << 30);
}

cudaError_t oz_gram_cols(OzSketch* o, const float* A32, const double* B, int64_t K, int64_t ld, int ell, double* C,
                         int64_t ldC, const char** why, cudaStream_t s, int* status, long long wait_cycles) {
  *why = nullptr;
  if (!tensor_map_encoder()) {
    *why = "cuTensorMapEncodeTiled unavailable";
    return cudaSuccess;
  }
  if ((ld % 32) || K < 1 || K > ld || ell < 1 || ldC < ell) {
    *why = "the operands' leading dimension must be a multiple of 32";
    return cudaSuccess;
  }
  cudaError_t e;
  const int64_t tot = ld * ell;
  const unsigned sg = (unsigned)std::min<int64_t>((tot + 255) / 256, 8192);
  if ((e = grow(&o->FD, &o->FD_b, (size_t)kDigZ * ell * ld * 2)) != cudaSuccess) return e;
  if ((e = grow(&o->fexp, &o->fexp_b, (size_t)ell * sizeof(int))) != cudaSuccess) return e;
  k_oz_colexp<double><<<(unsigned)ell, 256, 0, s>>>(B, ld, K, o->fexp);
  note_launch();
  k_oz_split_cols<double, kDigZ><<<sg, 256, 0, s>>>(B, ld, ell, o->fexp, o->FD);
  note_launch();
  CUtensorMap mA, mB;
  // the maps' K extent is K itself: rows K..ld-1 of the operands are read as zeros
  if (!make_tile_map(&mB, o->FD, 2, ell, K, ld, kDigZ, (int64_t)ell * ld, kBN)) {
    *why = "tensor map encoding failed";
    return cudaSuccess;
  }
  if (!A32) {
    // B^T B: both operands are B's planes
    if (!make_tile_map(&mA, o->FD, 2, ell, K, ld, kDigZ, (int64_t)ell * ld, kBM)) {
      *why = "tensor map encoding failed";
      return cudaSuccess;
    }
    return run_digit_gemm<kDigZ, kDigZ, 3>(o, mA, mB, ell, ell, K, o->fexp, o->fexp, nullptr, C, ldC, status, s,
                                           wait_cycles, true, 1 << 30);
  }
  if ((e = grow(&o->OD, &o->OD_b, (size_t)kDigOm * ell * ld * 2)) != cudaSuccess) return e;
  if ((e = grow(&o->oexp, &o->oexp_b, (size_t)ell * sizeof(int))) != cudaSuccess) return e;
  k_oz_colexp<float><<<(unsigned)ell, 256, 0, s>>>(A32, ld, K, o->oexp);
  note_launch();
  k_oz_split_cols<float, kDigOm><<<sg, 256, 0, s>>>(A32, ld, ell, o->oexp, o->OD);
  note_launch();
  if (!make_tile_map(&mA, o->OD, 2, ell, K, ld, kDigOm, (int64_t)ell * ld, kBM)) {
    *why = "tensor map encoding failed";
    return cudaSuccess;
  }
  return run_digit_gemm<kDigOm, kDigZ, 3>(o, mA, mB, ell, ell, K, o->oexp, o->fexp, nullptr, C, ldC, status, s,
                                          wait_cycles, true, 1 << 30);
}

cudaError_t oz_gemm_bw(OzSketch* o, const double* B, int64_t ldB, int64_t p, int ell, const double* W, int64_t ldW,
                       const double* colscale, double* U, int64_t ldU, const char** why, cudaStream_t s, int* status,
                       long long wait_cycles) {
  *why = nullptr;
  if (!tensor_map_encoder()) {
    *why = "cuTensorMapEncodeTiled unavailable";
    return cudaSuccess;
  }
  if (p < 1 || ell < 1 || ldU < p) {
    *why = "empty operands";
    return cudaSuccess;
  }
  const int64_t ldK = rup(ell, 32);
  cudaError_t e;
  if ((e = grow(&o->UA, &o->UA_b, (size_t)kDigZ * p * ldK * 2)) != cudaSuccess) return e;
  if ((e = grow(&o->UB, &o->UB_b, (size_t)kDigZ * ell * ldK * 2)) != cudaSuccess) return e;
  if ((e = grow(&o->uexp, &o->uexp_b, (size_t)p * sizeof(int))) != cudaSuccess) return e;
  if ((e = grow(&o->wexp, &o->wexp_b, (size_t)ell * sizeof(int))) != cudaSuccess) return e;
  if ((e = grow(&o->Ws, &o->Ws_b, (size_t)ell * ldK * sizeof(double))) != cudaSuccess) return e;
  k_oz_rowexp_cm<<<(unsigned)((p + 31) / 32), dim3(32, 8), 0, s>>>(B, ldB, p, ell, o->uexp);
  note_launch();
  {
    dim3 blk(32, 8), grd((unsigned)((p + 31) / 32), (unsigned)(ldK / 32));
    k_oz_split_rows_cm<<<grd, blk, 0, s>>>(B, ldB, p, ell, o->uexp, o->UA, ldK);
    note_launch();
  }
  {
    const int64_t tot = (int64_t)ell * ldK;
    k_oz_scale_pad<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(W, ldW, ell, ell, colscale, o->Ws, ldK);
    note_launch();
    k_oz_colexp<double><<<(unsigned)ell, 256, 0, s>>>(o->Ws, ldK, ell, o->wexp);
    note_launch();
    k_oz_split_cols<double, kDigZ><<<(unsigned)std::min<int64_t>((tot + 255) / 256, 8192), 256, 0, s>>>(
        o->Ws, ldK, ell, o->wexp, o->UB);
    note_launch();
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  CUtensorMap mA, mB;
  if (!make_tile_map(&mA, o->UA, 2, p, ldK, ldK, kDigZ, p * ldK, kBM) ||
      !make_tile_map(&mB, o->UB, 2, ell, ldK, ldK, kDigZ, (int64_t)ell * ldK, kBN)) {
    *why = "tensor map encoding failed";
    return cudaSuccess;
  }
  return run_digit_gemm<kDigZ, kDigZ, 3>(o, mA, mB, p, ell, ldK, o->uexp, o->wexp, nullptr, U, ldU, status, s,
                                         wait_cycles, false, 1 << 30);
}

cudaError_t oz_gram_self32(OzSketch* o, const float* A, int64_t K, int64_t ld, int ell, double* C, int64_t ldC,
                           const char** why, cudaStream_t s, int* status, long long wait_cycles) {
  *why = nullptr;
  if (!tensor_map_encoder()) {
    *why = "cuTensorMapEncodeTiled unavailable";
    return cudaSuccess;
  }
  if ((ld % 32) || K < 1 || K > ld || ell < 1 || ldC < ell) {
    *why = "the operand's leading dimension must be a multiple of 32";
    return cudaSuccess;
  }
  cudaError_t e;
  const int64_t tot = ld * ell;
  if ((e = grow(&o->OD, &o->OD_b, (size_t)kDigOm * ell * ld * 2)) != cudaSuccess) return e;
  if ((e = grow(&o->oexp, &o->oexp_b, (size_t)ell * sizeof(int))) != cudaSuccess) return e;
  k_oz_colexp<float><<<(unsigned)ell, 256, 0, s>>>(A, ld, K, o->oexp);
  note_launch();
  k_oz_split_cols<float, kDigOm><<<(unsigned)std::min<int64_t>((tot + 255) / 256, 8192), 256, 0, s>>>(A, ld, ell,
                                                                                                    o->oexp, o->OD);
  note_launch();
  CUtensorMap mA, mB;
  if (!make_tile_map(&mA, o->OD, 2, ell, K, ld, kDigOm, (int64_t)ell * ld, kBM) ||
      !make_tile_map(&mB, o->OD, 2, ell, K, ld, kDigOm, (int64_t)ell * ld, kBN)) {
    *why = "tensor map encoding failed";
    return cudaSuccess;
  }
  return run_digit_gemm<kDigOm, kDigOm, 3>(o, mA, mB, ell, ell, K, o->oexp, o->oexp, nullptr, C, ldC, status, s,
                                           wait_cycles, true, 1 << 30);
}

cudaError_t oz_syrk_sub(OzSketch* o, const double* P, int64_t ldP, int64_t m, int bs, double* C, int64_t ldC,
                        const char** why, cudaStream_t s, int* status, long long wait_cycles) {
  *why = nullptr;
  if (!tensor_map_encoder()) {
    *why = "cuTensorMapEncodeTiled unavailable";
    return cudaSuccess;
  }
  if (m < 1 || bs < 1 || bs > kChunk) {
    *why = "the panel must be 1 to 256 columns wide";
    return cudaSuccess;
  }
  const int64_t ldK = rup(bs, 32);
  cudaError_t e;
  if ((e = grow(&o->UA, &o->UA_b, (size_t)kDigZ * m * ldK * 2)) != cudaSuccess) return e;
  if ((e = grow(&o->uexp, &o->uexp_b, (size_t)m * sizeof(int))) != cudaSuccess) return e;
  k_oz_rowexp_cm<<<(unsigned)((m + 31) / 32), dim3(32, 8), 0, s>>>(P, ldP, m, bs, o->uexp);
  note_launch();
  {
    dim3 blk(32, 8), grd((unsigned)((m + 31) / 32), (unsigned)(ldK / 32));
    k_oz_split_rows_cm<<<grd, blk, 0, s>>>(P, ldP, m, bs, o->uexp, o->UA, ldK);
    note_launch();
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  CUtensorMap mA, mB;
  if (!make_tile_map(&mA, o->UA, 2, m, ldK, ldK, kDigZ, m * ldK, kBM) ||
      !make_tile_map(&mB, o->UA, 2, m, ldK, ldK, kDigZ, m * ldK, kBN)) {
    *why = "tensor map encoding failed";
    return cudaSuccess;
  }
  // one K chunk: each lower tile summed by one CTA and subtracted from C by the epilogue
  return run_digit_gemm<kDigZ, kDigZ, 3>(o, mA, mB, m, m, ldK, o->uexp, o->uexp, nullptr, C, ldC, status, s,
                                         wait_cycles, true, 1 << 30, kPartialCap, true);
}

}  // namespace ngd
