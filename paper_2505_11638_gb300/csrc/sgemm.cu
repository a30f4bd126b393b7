// FP32 SIMT GEMM for the layer products of the matrix-free Jacobian products (vjp_rev.cu):
// C(m, n) = sum_k A(m, k) B(k, n) with arbitrary element strides (either operand may have its
// unit stride along k or along m / n), FP32 accumulation over one K-slice per CTA (blockIdx.z,
// at most kMaxSlice terms, so that the rounding stays near 2^-24 sqrt(slice) of the terms), the
// slice result written as an FP64 partial (out64 + z * split_stride) or, for a single slice, to
// an FP32 output (optionally added to it).
//
// 128 x 128 tile per CTA of 256 threads, 8 x 8 outputs per thread taken as four 4 x 4 quadrants
// (rows ty*4 .. +3 and 64 + ty*4 .. +3, likewise columns) so that the shared-memory reads of a k
// step are four float4 loads per thread; 16-deep K tiles, double-buffered in shared memory with
// the next tile's global loads issued before the current tile's arithmetic.
#include <cuda_runtime.h>

#include <algorithm>

#include "df.cuh"
#include "linalg.cuh"

namespace ngd {

namespace {

constexpr int TM = 128, TN = 128, TK = 16;

__global__ void __launch_bounds__(256) k_sgemm(int64_t M, int64_t N, int64_t K, const float* __restrict__ A,
                                               int64_t sam, int64_t sak, const float* __restrict__ B, int64_t sbk,
                                               int64_t sbn, int64_t kps, double* __restrict__ out64,
                                               int64_t split_stride, float* __restrict__ outT, int64_t scm,
                                               int64_t scn, int accumulate) {
  __shared__ __align__(16) float As[2][TK][TM + 4];
  __shared__ __align__(16) float Bs[2][TK][TN + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t m0 = (int64_t)blockIdx.x * TM, n0 = (int64_t)blockIdx.y * TN;
  const int64_t kb = (int64_t)blockIdx.z * kps, ke = min(K, kb + kps);
  // global load pattern: 8 elements of A and 8 of B per thread per K tile, consecutive threads on
  // the unit-stride dimension
  float ra[8], rb[8];
  auto load = [&](int64_t k0) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = tid + 256 * q;
      int mm, kk;
      if (sak == 1) { kk = e % TK; mm = e / TK; } else { mm = e % TM; kk = e / TM; }
      const int64_t gm = m0 + mm, gk = k0 + kk;
      ra[q] = (gm < M && gk < ke) ? A[gm * sam + gk * sak] : 0.0f;
      int nn, kk2;
      if (sbk == 1) { kk2 = e % TK; nn = e / TK; } else { nn = e % TN; kk2 = e / TN; }
      const int64_t gn = n0 + nn, gk2 = k0 + kk2;
      rb[q] = (gn < N && gk2 < ke) ? B[gk2 * sbk + gn * sbn] : 0.0f;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = tid + 256 * q;
      int mm, kk;
      if (sak == 1) { kk = e % TK; mm = e / TK; } else { mm = e % TM; kk = e / TM; }
      As[buf][kk][mm] = ra[q];
      int nn, kk2;
      if (sbk == 1) { kk2 = e % TK; nn = e / TK; } else { nn = e % TN; kk2 = e / TN; }
      Bs[buf][kk2][nn] = rb[q];
    }
  };
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
  int buf = 0;
  if (kb < ke) {
    load(kb);
    store(0);
  }
  __syncthreads();
  for (int64_t k0 = kb; k0 < ke; k0 += TK) {
    const bool more = k0 + TK < ke;
    if (more) load(k0 + TK);
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + tx * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (more) store(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t gm = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int64_t gn = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
      if (gn >= N) continue;
      if (out64) {
        out64[(int64_t)blockIdx.z * split_stride + gm * scm + gn * scn] = f32_to_f64(acc[i][j]);
      } else {
        float* o = outT + gm * scm + gn * scn;
        *o = accumulate ? *o + acc[i][j] : acc[i][j];
      }
    }
  }
}

}  // namespace

int sgemm_layer_slices(int64_t M, int64_t N, int64_t K) {
  constexpr int64_t kMaxSlice = 1024;
  const int64_t tiles = ((M + TM - 1) / TM) * ((N + TN - 1) / TN);
  int64_t ns = (K + kMaxSlice - 1) / kMaxSlice;
  // more slices while the tiles alone leave SMs idle (K-slices of at least 256 terms)
  while (tiles * ns < 300 && K / (ns + 1) >= 256) ++ns;
  ns = std::max<int64_t>(1, ns);
  const int64_t kps = ((K + ns - 1) / ns + TK - 1) / TK * TK;     // as launch_sgemm_layer cuts K
  return (int)std::max<int64_t>(1, (K + kps - 1) / kps);
}

void launch_sgemm_layer(const GemmArgs<float>& g, int nslices, cudaStream_t s) {
  const int64_t kps = ((g.K + nslices - 1) / nslices + TK - 1) / TK * TK;
  const int nz = (int)std::max<int64_t>(1, (g.K + kps - 1) / kps);
  dim3 grid((unsigned)((g.M + TM - 1) / TM), (unsigned)((g.N + TN - 1) / TN), (unsigned)nz);
  k_sgemm<<<grid, 256, 0, s>>>(g.M, g.N, g.K, g.A, g.sam, g.sak, g.B, g.sbk, g.sbn, kps, g.out64, g.split_stride,
                               g.outT, g.scm, g.scn, g.accumulate);
  note_launch();
}

}  // namespace ngd
