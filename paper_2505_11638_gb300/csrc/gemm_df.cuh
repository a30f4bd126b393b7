// The double-float GEMM's templates: FP64-accurate products on the FP32 pipes (k_gemm_df for any
// strides, k_gemm_dfv for 16-byte-aligned tiles, 128 x 64 or 128 x 32 block tiles), with optional
// K slices, row / column scales, accumulation and lower-triangle output.  Each operand-type pair is
// instantiated in a translation unit of its own (gemm_df_<types>.cu), so that they compile in
// parallel.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "df.cuh"
#include "linalg.cuh"

namespace ngd {

// ---------------------------------------------------------------------------- double-float GEMM
// FP64-accurate C(m,n) = sum_k A(m,k) B(k,n) on the FP32 pipes (same strides as k_gemm).  Float
// operands are exact FP32 values; double operands are split into FP32 hi + lo on load.  Every
// product hi*hi is made exact with fmaf and summed by TwoSum; the cross terms hi*lo, lo*hi go
// into the low word.  Relative accuracy ~2^-44 per term, at ~10-14 FP32 operations per
// multiply-add instead of one FMA on the scarce FP64 units.
template <typename T> struct IsDouble { static constexpr bool v = false; };
template <> struct IsDouble<double> { static constexpr bool v = true; };

template <typename TA, typename TB>
__global__ void __launch_bounds__(256) k_gemm_df(int64_t M, int64_t N, int64_t K, const TA* __restrict__ A,
                                                 int64_t sam, int64_t sak, const TB* __restrict__ B, int64_t sbk,
                                                 int64_t sbn, int64_t k_per_split, double* __restrict__ out64,
                                                 int64_t split_stride, float* __restrict__ out32, int64_t scm,
                                                 int64_t scn, const double* __restrict__ rowscale,
                                                 const double* __restrict__ colscale, int accumulate, int lower) {
  constexpr int BM = 64, BN = 64, BK = 16;
  constexpr bool AL = IsDouble<TA>::v, BL = IsDouble<TB>::v;
  __shared__ float Ah[BK][BM + 1];
  __shared__ float Al[AL ? BK : 1][AL ? BM + 1 : 1];
  __shared__ float Bh[BK][BN + 1];
  __shared__ float Bl[BL ? BK : 1][BL ? BN + 1 : 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;
  if (lower && n0 >= m0 + BM) return;                      // tile wholly above the diagonal
  const int64_t kb = (int64_t)blockIdx.z * k_per_split;
  const int64_t ke = min(K, kb + k_per_split);
  DF acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = DF{0.f, 0.f};
  for (int64_t k0 = kb; k0 < ke; k0 += BK) {
    for (int e = threadIdx.x; e < BM * BK; e += 256) {
      int mm, kk;
      if (sak == 1) { kk = e % BK; mm = e / BK; } else { mm = e % BM; kk = e / BM; }
      const int64_t gm = m0 + mm, gk = k0 + kk;
      const TA x = (gm < M && gk < ke) ? A[gm * sam + gk * sak] : TA(0);
      if constexpr (AL) {
        float h, l;
        split_df((double)x, h, l);
        Ah[kk][mm] = h;
        Al[kk][mm] = l;
      } else {
        Ah[kk][mm] = (float)x;
      }
    }
    for (int e = threadIdx.x; e < BK * BN; e += 256) {
      int kk, nn;
      if (sbk == 1) { kk = e % BK; nn = e / BK; } else { nn = e % BN; kk = e / BN; }
      const int64_t gk = k0 + kk, gn = n0 + nn;
      const TB x = (gn < N && gk < ke) ? B[gk * sbk + gn * sbn] : TB(0);
      if constexpr (BL) {
        float h, l;
        split_df((double)x, h, l);
        Bh[kk][nn] = h;
        Bl[kk][nn] = l;
      } else {
        Bh[kk][nn] = (float)x;
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < BK; ++kk) {
      float ah[4], bh[4], al[4], bl[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        ah[i] = Ah[kk][ty + 16 * i];
        bh[i] = Bh[kk][tx + 16 * i];
        al[i] = AL ? Al[kk][ty + 16 * i] : 0.f;
        bl[i] = BL ? Bl[kk][tx + 16 * i] : 0.f;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          DF& s = acc[i][j];
          const float p = ah[i] * bh[j];
          float lo = fmaf(ah[i], bh[j], -p);           // exact error of the product
          if constexpr (BL) lo = fmaf(ah[i], bl[j], lo);
          if constexpr (AL) lo = fmaf(al[i], bh[j], lo);
          const float t = s.hi + p;                    // TwoSum(s.hi, p)
          const float z = t - s.hi;
          s.lo += ((s.hi - (t - z)) + (p - z)) + lo;
          s.hi = t;
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
    const double rs = rowscale ? rowscale[gm] : 1.0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t gn = n0 + tx + 16 * j;
      if (gn >= N || (lower && gn > gm)) continue;
      double v = (f32_to_f64(acc[i][j].hi) + f32_to_f64(acc[i][j].lo)) * rs;
      if (colscale) v *= colscale[gn];
      if (out64) {
        double* o = out64 + (int64_t)blockIdx.z * split_stride + gm * scm + gn * scn;
        *o = accumulate ? *o + v : v;
      } else {
        float* o = out32 + gm * scm + gn * scn;
        *o = accumulate ? (float)((double)*o + v) : (float)v;
      }
    }
  }
}

// Double-float GEMM for operands whose tiles load as 16-byte vectors: A either K-contiguous
// (sak = 1) or M-contiguous (sam = 1), B either K-contiguous (sbk = 1) or N-contiguous (sbn = 1).
// Same arithmetic and epilogue as k_gemm_df (exact FP32 products, TwoSum accumulation, FP64
// outputs), on a 128 x 64 block tile, K in steps of 16.  Thread (ty, tx) owns rows
// 4 ty .. 4 ty + 3 and 64 + 4 ty .. 64 + 4 ty + 3 and columns 4 tx .. 4 tx + 3; rows are paired so
// that each pair is one f32x2 register and one multiply-add instruction covers two outputs.
// Shared memory holds A and B as [k][m] and [k][n] (high words, and low words of FP64 inputs) in
// two stages; the next K step is loaded into registers while the current one is multiplied.
namespace gdf {
constexpr int BM = 128, BN = 64, BK = 16, NT = 256;
constexpr int LA = BM + 4, LB = BN + 4;          // row lengths in shared memory (16-byte multiples)

template <bool AL, bool BL>
__device__ __forceinline__ void mac2(DF2& s, f2x ah, f2x nah, f2x al, f2x bh, f2x bl) {
  const f2x pn = mul2(nah, bh);                  // -(ah bh), rounded; its error is one fma
  const f2x pe = fma2(ah, bh, pn);
  const f2x t = sub2(s.hi, pn);                  // TwoSum(s.hi, ah bh)
  const f2x z = sub2(t, s.hi);
  const f2x e = sub2(sub2(s.hi, sub2(t, z)), add2(pn, z));
  f2x lo = s.lo;
  if constexpr (BL) lo = fma2(ah, bl, lo);
  if constexpr (AL) lo = fma2(al, bh, lo);
  s.hi = t;
  s.lo = add2(add2(lo, pe), e);
}

// Register staging of one K step: A (BM x BK) and B (BK x BN) elements this thread loads.
template <typename T, bool KC, int ROWS>
struct Stage {
  // KC: the tile's contiguous direction is K (ROWS = m or n rows of BK contiguous values);
  // otherwise it is the ROWS direction (BK rows of ROWS contiguous values).
  static constexpr int V = 16 / sizeof(T);                 // elements per 16-byte vector
  static constexpr int NV = ROWS * BK / V / NT;            // vectors per thread
  T v[NV][V];
  __device__ __forceinline__ void load(const T* __restrict__ X, int64_t srow, int64_t scol, int64_t r0, int64_t k0,
                                       int64_t R, int64_t ke, bool interior) {
    const int t = threadIdx.x;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const int e = t + i * NT;                            // vector index within the tile
      int rr, kk;
      if (KC) { rr = e / (BK / V); kk = (e % (BK / V)) * V; }
      else { kk = e / (ROWS / V); rr = (e % (ROWS / V)) * V; }
      const int64_t gr = r0 + rr, gk = k0 + kk;
      if (interior) {
        const T* src = KC ? X + gr * srow + gk : X + gk * scol + gr;
        if constexpr (sizeof(T) == 4) {
          const float4 q = __ldg(reinterpret_cast<const float4*>(src));
          v[i][0] = q.x; v[i][1] = q.y; v[i][2] = q.z; v[i][3] = q.w;
        } else {
          const double2 q = __ldg(reinterpret_cast<const double2*>(src));
          v[i][0] = q.x; v[i][1] = q.y;
        }
      } else {
#pragma unroll
        for (int u = 0; u < V; ++u) {
          const int64_t r = KC ? gr : gr + u, k = KC ? gk + u : gk;
          v[i][u] = (r < R && k < ke) ? (KC ? X[r * srow + k] : X[k * scol + r]) : T(0);
        }
      }
    }
  }
  // into shared memory as [k][row] (row length L), high words in hi, low words of FP64 in lo
  template <int L>
  __device__ __forceinline__ void store(float* hi, float* lo) const {
    const int t = threadIdx.x;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const int e = t + i * NT;
      int rr, kk;
      if (KC) { rr = e / (BK / V); kk = (e % (BK / V)) * V; }
      else { kk = e / (ROWS / V); rr = (e % (ROWS / V)) * V; }
#pragma unroll
      for (int u = 0; u < V; ++u) {
        const int r = KC ? rr : rr + u, k = KC ? kk + u : kk;
        if constexpr (sizeof(T) == 8) {
          float h, l;
          split_df((double)v[i][u], h, l);
          hi[k * L + r] = h;
          lo[k * L + r] = l;
        } else {
          hi[k * L + r] = (float)v[i][u];
        }
      }
    }
  }
};

template <typename TA, typename TB, bool AKC, bool BKC, int TN>
__global__ void __launch_bounds__(NT, 2) k_gemm_dfv(int64_t M, int64_t N, int64_t K, const TA* __restrict__ A,
                                                    int64_t sam, int64_t sak, const TB* __restrict__ B, int64_t sbk,
                                                    int64_t sbn, int64_t k_per_split, double* __restrict__ out64,
                                                    int64_t split_stride, float* __restrict__ out32, int64_t scm,
                                                    int64_t scn, const double* __restrict__ rowscale,
                                                    const double* __restrict__ colscale, int accumulate,
                                                    int lower) {
  constexpr bool AL = IsDouble<TA>::v, BL = IsDouble<TB>::v;
  static_assert(TN == BN || TN == BN / 2, "tile width");
  constexpr int LBt = TN + 4;                               // B row length in shared memory
  constexpr int TXN = TN / 4;                               // threads along n
  constexpr int RP = BM / (NT / TXN) / 2;                   // row pairs per thread: 4 (TN 64) or 2 (TN 32)
  constexpr int SA = BK * LA, SB = BK * LBt;                // floats per stage and word
  extern __shared__ __align__(16) float sh[];
  float* Ah = sh;                                           // [2][BK][LA]
  float* Al = Ah + 2 * SA;                                  // [2][BK][LA] when AL
  float* Bh = Al + (AL ? 2 * SA : 0);                       // [2][BK][LBt]
  float* Bl = Bh + 2 * SB;                                  // [2][BK][LBt] when BL
  const int tx = threadIdx.x % TXN, ty = threadIdx.x / TXN;
  const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * TN;
  if (lower && n0 >= m0 + BM) return;                      // tile wholly above the diagonal
  const int64_t kb = (int64_t)blockIdx.z * k_per_split;
  const int64_t ke = min(K, kb + k_per_split);
  const bool mn_in = m0 + BM <= M && n0 + TN <= N;
  DF2 acc[RP][4];
#pragma unroll
  for (int i = 0; i < RP; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = DF2{0ull, 0ull};
  Stage<TA, AKC, BM> sa;
  Stage<TB, BKC, TN> sb;
  const int nk = (int)((ke - kb + BK - 1) / BK);
  if (nk > 0) {
    const bool in0 = mn_in && kb + BK <= ke;
    sa.load(A, AKC ? sam : 0, AKC ? 0 : sak, m0, kb, M, ke, in0);
    sb.load(B, BKC ? sbn : 0, BKC ? 0 : sbk, n0, kb, N, ke, in0);
    sa.template store<LA>(Ah, Al);
    sb.template store<LBt>(Bh, Bl);
  }
  __syncthreads();
  for (int it = 0; it < nk; ++it) {
    const int cur = it & 1;
    const int64_t kn = kb + (int64_t)(it + 1) * BK;
    if (it + 1 < nk) {                                      // next K step into registers
      const bool in = mn_in && kn + BK <= ke;
      sa.load(A, AKC ? sam : 0, AKC ? 0 : sak, m0, kn, M, ke, in);
      sb.load(B, BKC ? sbn : 0, BKC ? 0 : sbk, n0, kn, N, ke, in);
    }
    const float* ah_s = Ah + cur * SA;
    const float* al_s = Al + cur * SA;
    const float* bh_s = Bh + cur * SB;
    const float* bl_s = Bl + cur * SB;
#pragma unroll 4
    for (int kk = 0; kk < BK; ++kk) {
      // rows 4 ty .. 4 ty + 3, and for TN 64 also 64 + 4 ty .. 64 + 4 ty + 3
      f2x ah[RP], al[RP];
#pragma unroll
      for (int h = 0; h < RP / 2; ++h) {
        const float4 a0 = *reinterpret_cast<const float4*>(ah_s + kk * LA + 64 * h + 4 * ty);
        ah[2 * h] = pk2(a0.x, a0.y);
        ah[2 * h + 1] = pk2(a0.z, a0.w);
        al[2 * h] = al[2 * h + 1] = 0ull;
        if constexpr (AL) {
          const float4 c0 = *reinterpret_cast<const float4*>(al_s + kk * LA + 64 * h + 4 * ty);
          al[2 * h] = pk2(c0.x, c0.y);
          al[2 * h + 1] = pk2(c0.z, c0.w);
        }
      }
      const float4 b0 = *reinterpret_cast<const float4*>(bh_s + kk * LBt + 4 * tx);
      const float bhv[4] = {b0.x, b0.y, b0.z, b0.w};
      float blv[4] = {0.f, 0.f, 0.f, 0.f};
      if constexpr (BL) {
        const float4 d0 = *reinterpret_cast<const float4*>(bl_s + kk * LBt + 4 * tx);
        blv[0] = d0.x; blv[1] = d0.y; blv[2] = d0.z; blv[3] = d0.w;
      }
#pragma unroll
      for (int i = 0; i < RP; ++i) {
        const f2x nah = ah[i] ^ 0x8000000080000000ull;
#pragma unroll
        for (int j = 0; j < 4; ++j) mac2<AL, BL>(acc[i][j], ah[i], nah, al[i], pk2(bhv[j], bhv[j]), pk2(blv[j], blv[j]));
      }
    }
    if (it + 1 < nk) {
      sa.template store<LA>(Ah + (cur ^ 1) * SA, Al + (cur ^ 1) * SA);
      sb.template store<LBt>(Bh + (cur ^ 1) * SB, Bl + (cur ^ 1) * SB);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < RP; ++i) {
    float h0, h1, l0, l1;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      upk2(acc[i][j].hi, h0, h1);
      upk2(acc[i][j].lo, l0, l1);
      const int64_t gn = n0 + 4 * tx + j;
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int64_t gm = m0 + 64 * (i / 2) + 4 * ty + 2 * (i % 2) + u;
        if (gm >= M || gn >= N || (lower && gn > gm)) continue;
        double v = f32_to_f64(u ? h1 : h0) + f32_to_f64(u ? l1 : l0);
        if (rowscale) v *= rowscale[gm];
        if (colscale) v *= colscale[gn];
        if (out64) {
          double* o = out64 + (int64_t)blockIdx.z * split_stride + gm * scm + gn * scn;
          *o = accumulate ? *o + v : v;
        } else {
          float* o = out32 + gm * scm + gn * scn;
          *o = accumulate ? f64_to_f32_rn(f32_to_f64(*o) + v) : f64_to_f32_rn(v);
        }
      }
    }
  }
}

template <typename TA, typename TB, int TN>
constexpr size_t smem_bytes() {
  return sizeof(float) * (2 * BK * LA * (IsDouble<TA>::v ? 2 : 1) + 2 * BK * (TN + 4) * (IsDouble<TB>::v ? 2 : 1));
}

template <typename TA, typename TB, bool AKC, bool BKC, int TN>
void launch_v(const GemmDfArgs<TA, TB>& g, int64_t kps, int nz, cudaStream_t s) {
  constexpr size_t smem = smem_bytes<TA, TB, TN>();
  auto kern = k_gemm_dfv<TA, TB, AKC, BKC, TN>;
  static bool configured = false;
  if (!configured) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    configured = true;
  }
  dim3 grid((unsigned)((g.M + BM - 1) / BM), (unsigned)((g.N + TN - 1) / TN), (unsigned)std::max(nz, 1));
  kern<<<grid, NT, smem, s>>>(g.M, g.N, g.K, g.A, g.sam, g.sak, g.B, g.sbk, g.sbn, kps, g.out64, g.split_stride,
                              g.out32, g.scm, g.scn, g.rowscale, g.colscale, g.accumulate, g.lower);
  note_launch();
}

inline bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }
}  // namespace gdf

template <typename TA, typename TB>
void launch_gemm_df(const GemmDfArgs<TA, TB>& g, cudaStream_t s) {
  const int64_t kps = g.nsplit > 1 ? ((g.K + g.nsplit - 1) / g.nsplit + 15) / 16 * 16 : std::max<int64_t>(g.K, 1);
  const int nz = (int)((g.K + kps - 1) / kps);
  // vectorised kernel when every 16-byte vector of a tile starts on a 16-byte boundary
  {
    constexpr int va = 16 / sizeof(TA), vb = 16 / sizeof(TB);
    const bool akc = g.sak == 1, amc = g.sam == 1 && !akc, bkc = g.sbk == 1, bnc = g.sbn == 1 && !bkc;
    const bool a_ok = gdf::aligned16(g.A) && ((akc && g.sam % va == 0) || (amc && g.sak % va == 0));
    const bool b_ok = gdf::aligned16(g.B) && ((bkc && g.sbn % vb == 0) || (bnc && g.sbk % vb == 0));
    if (a_ok && b_ok && g.M > 0 && g.N > 0) {
      // outputs at most 32 wide (the column blocks of RPCholesky, early low-rank sketches) on the
      // 128 x 32 tile when B is FP64 (one 16-byte vector per thread and K step)
      if constexpr (sizeof(TB) == 8) {
        if (g.N <= gdf::BN / 2) {
          if (akc && bkc) return gdf::launch_v<TA, TB, true, true, gdf::BN / 2>(g, kps, nz, s);
          if (akc && bnc) return gdf::launch_v<TA, TB, true, false, gdf::BN / 2>(g, kps, nz, s);
          if (amc && bkc) return gdf::launch_v<TA, TB, false, true, gdf::BN / 2>(g, kps, nz, s);
          return gdf::launch_v<TA, TB, false, false, gdf::BN / 2>(g, kps, nz, s);
        }
      }
      if (akc && bkc) return gdf::launch_v<TA, TB, true, true, gdf::BN>(g, kps, nz, s);
      if (akc && bnc) return gdf::launch_v<TA, TB, true, false, gdf::BN>(g, kps, nz, s);
      if (amc && bkc) return gdf::launch_v<TA, TB, false, true, gdf::BN>(g, kps, nz, s);
      return gdf::launch_v<TA, TB, false, false, gdf::BN>(g, kps, nz, s);
    }
  }
  dim3 grid((unsigned)((g.M + 63) / 64), (unsigned)((g.N + 63) / 64), (unsigned)std::max(nz, 1));
  k_gemm_df<TA, TB><<<grid, 256, 0, s>>>(g.M, g.N, g.K, g.A, g.sam, g.sak, g.B, g.sbk, g.sbn, kps, g.out64,
                                         g.split_stride, g.out32, g.scm, g.scn, g.rowscale, g.colscale,
                                         g.accumulate, g.lower); note_launch();
}

}  // namespace ngd
