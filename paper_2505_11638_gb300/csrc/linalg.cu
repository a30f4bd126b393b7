// Dense kernels of the NGD hot path: deterministic reductions, the stored-Jacobian
// Gramian matvec, preconditioned-CG vector updates, the Nystrom preconditioner, the
// Philox Gaussian test matrix, a tiled SIMT GEMM (FP64 / FP32 with FP64 cross-tile
// sums), the row-wise triangular solve and the FP64 blocked Cholesky of the l x l core.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math_constants.h>

#include <algorithm>

#include "df.cuh"
#include "linalg.cuh"
#include "sketch_oz.cuh"

namespace cg = cooperative_groups;

namespace ngd {

template <typename T> __device__ __forceinline__ T wsum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of one double per thread (blockDim.x a multiple of 32, <= 1024).
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = wsum(v);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  }
  return s;  // valid in thread 0
}

// "Last block finishes" reduction: each block stores its partial; the block that
// arrives last sums all partials in block order (deterministic) and returns true in
// thread 0 with the total in *total.
__device__ __forceinline__ bool last_block_total(double mine, double* part, unsigned int* counter, double* total) {
  __shared__ bool is_last;
  if (threadIdx.x == 0) {
    part[blockIdx.x] = mine;
    __threadfence();
    const unsigned int prev = atomicAdd(counter, 1u);
    is_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return false;
  if (threadIdx.x == 0) {
    __threadfence();
    double s = 0.0;
    volatile double* vp = part;
    for (unsigned int b = 0; b < gridDim.x; ++b) s += vp[b];
    *total = s;
    *counter = 0u;
  }
  return threadIdx.x == 0;
}

// ---------------------------------------------------------------------------- reductions
__global__ void k_sum_partials(const double* __restrict__ part, int n, double scale, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  // fixed assignment of partials to threads, fixed tree: deterministic
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) *out = s * scale;
}

void launch_sum_partials(const double* part, int n, double scale, double* out, cudaStream_t s) {
  k_sum_partials<<<1, 256, 0, s>>>(part, n, scale, out); note_launch();
}

// ---------------------------------------------------------------------------- conversions
template <typename T>
__global__ void k_d2t(const double* __restrict__ x, T* __restrict__ y, int64_t n, int64_t npad) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npad; i += stride)
    y[i] = i < n ? (T)x[i] : T(0);
}

template <typename T>
void launch_d2t(const double* x, T* y, int64_t n, int64_t npad, cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>((npad + 255) / 256, 2048);
  k_d2t<T><<<blocks, 256, 0, s>>>(x, y, n, npad); note_launch();
}
template void launch_d2t<float>(const double*, float*, int64_t, int64_t, cudaStream_t);
template void launch_d2t<double>(const double*, double*, int64_t, int64_t, cudaStream_t);


// ---------------------------------------------------------------------------- stored-J matvec
// t[n] = sum_j J[n, j] v[j] (v already in the working dtype, zero-padded to ldJ),
// s[n] = w[n] t[n].  One warp per row, 16-byte vector loads.
template <typename T> struct Vec;
template <> struct Vec<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec<double> { using type = double2; static constexpr int n = 2; };

template <typename T>
__device__ __forceinline__ T vdot(const typename Vec<T>::type& a, const typename Vec<T>::type& b);
template <> __device__ __forceinline__ float vdot<float>(const float4& a, const float4& b) {
  return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
}
template <> __device__ __forceinline__ double vdot<double>(const double2& a, const double2& b) {
  return a.x * b.x + a.y * b.y;
}

template <typename T>
__global__ void __launch_bounds__(256) k_rowdot(const T* __restrict__ J, int64_t ldJ, int64_t nrows,
                                                const T* __restrict__ v, const double* __restrict__ w,
                                                double* __restrict__ t_out, double* __restrict__ s_out,
                                                const int* __restrict__ done) {
  if (done && *done) return;
  using V = typename Vec<T>::type;
  constexpr int VN = Vec<T>::n;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t nv = ldJ / VN;
  const V* __restrict__ vv = reinterpret_cast<const V*>(v);
  for (int64_t row = warp; row < nrows; row += nwarps) {
    const V* __restrict__ jr = reinterpret_cast<const V*>(J + row * ldJ);
    T a0 = T(0), a1 = T(0);
    int64_t k = lane;
    for (; k + 32 < nv; k += 64) {
      a0 += vdot<T>(jr[k], vv[k]);
      a1 += vdot<T>(jr[k + 32], vv[k + 32]);
    }
    if (k < nv) a0 += vdot<T>(jr[k], vv[k]);
    const double tsum = (double)wsum(a0 + a1);
    if (lane == 0) {
      if (t_out) t_out[row] = tsum;
      if (s_out) s_out[row] = w ? w[row] * tsum : tsum;
    }
  }
}

template <typename T>
void launch_rowdot(const T* J, int64_t ldJ, int64_t nrows, const T* v, const double* w, double* t_out,
                   double* s_out, const int* done, cudaStream_t s) {
  const int64_t warps = nrows;
  const int blocks = (int)std::min<int64_t>((warps * 32 + 255) / 256, 152 * 16);
  k_rowdot<T><<<blocks, 256, 0, s>>>(J, ldJ, nrows, v, w, t_out, s_out, done); note_launch();
}
template void launch_rowdot<float>(const float*, int64_t, int64_t, const float*, const double*, double*, double*,
                                   const int*, cudaStream_t);
template void launch_rowdot<double>(const double*, int64_t, int64_t, const double*, const double*, double*,
                                    double*, const int*, cudaStream_t);

// part[split][j] = sum_{rows of split} J[n, j] s[n]; each thread owns VN consecutive columns.
template <typename T>
__global__ void __launch_bounds__(256) k_coldot(const T* __restrict__ J, int64_t ldJ, int64_t nrows,
                                                const double* __restrict__ s, double* __restrict__ part,
                                                int64_t rows_per_split, const int* __restrict__ done) {
  if (done && *done) return;
  using V = typename Vec<T>::type;
  constexpr int VN = Vec<T>::n;
  const int64_t col = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * VN;
  if (col >= ldJ) return;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_split;
  const int64_t r1 = min(nrows, r0 + rows_per_split);
  T acc[VN];
#pragma unroll
  for (int e = 0; e < VN; ++e) acc[e] = T(0);
  for (int64_t n = r0; n < r1; ++n) {
    const T sn = (T)s[n];
    const V jv = *reinterpret_cast<const V*>(J + n * ldJ + col);
    const T* je = reinterpret_cast<const T*>(&jv);
#pragma unroll
    for (int e = 0; e < VN; ++e) acc[e] += je[e] * sn;
  }
  double* pp = part + (int64_t)blockIdx.y * ldJ + col;
#pragma unroll
  for (int e = 0; e < VN; ++e) pp[e] = to_f64(acc[e]);
}

int coldot_nsplit(int64_t nrows, int64_t ldJ, int vn) {
  const int64_t colblocks = (ldJ / vn + 255) / 256;
  int64_t ns = std::max<int64_t>(1, 1216 / std::max<int64_t>(colblocks, 1));
  ns = std::min<int64_t>(ns, std::max<int64_t>(1, nrows / 16));
  return (int)std::min<int64_t>(ns, 1024);
}

template <typename T>
void launch_coldot(const T* J, int64_t ldJ, int64_t nrows, const double* s_vec, double* part, int nsplit,
                   const int* done, cudaStream_t st) {
  constexpr int VN = Vec<T>::n;
  const int64_t rps = (nrows + nsplit - 1) / nsplit;
  dim3 grid((unsigned)((ldJ / VN + 255) / 256), (unsigned)nsplit);
  k_coldot<T><<<grid, 256, 0, st>>>(J, ldJ, nrows, s_vec, part, rps, done); note_launch();
}
template void launch_coldot<float>(const float*, int64_t, int64_t, const double*, double*, int, const int*,
                                   cudaStream_t);
template void launch_coldot<double>(const double*, int64_t, int64_t, const double*, double*, int, const int*,
                                    cudaStream_t);

// FP32 Jacobian with FP64-accurate sums.  In the directions of G's small eigenvalues the
// matvec is a sum of terms that cancel to ~mu / lambda_1 of their size (1e-9 for the 5-D
// Poisson workload after a few steps), so FP32 accumulation noise (~1e-7 of the terms) hides
// those directions from CG and it stalls.  Each FP32 product is made exact with fmaf and the
// products are summed as double-float pairs (TwoSum), which costs ~11 FP32 operations per
// Jacobian element and keeps the kernels bound by HBM, not by the scarce FP64 units.
__global__ void k_split_df(const double* __restrict__ x, float* __restrict__ hi, float* __restrict__ lo, int64_t n,
                           int64_t npad) {
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npad; i += st) {
    float h = 0.f, l = 0.f;
    if (i < n) split_df(x[i], h, l);
    hi[i] = h;
    lo[i] = l;
  }
}
__global__ void k_f64_to_f32(const double* __restrict__ x, float* __restrict__ y, int64_t n) {
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += st) y[i] = f64_to_f32_rn(x[i]);
}
void launch_f64_to_f32(const double* x, float* y, int64_t n, cudaStream_t s) {
  k_f64_to_f32<<<(int)std::min<int64_t>((n + 255) / 256, 2048), 256, 0, s>>>(x, y, n); note_launch();
}

void launch_split_df(const double* x, float* hi, float* lo, int64_t n, int64_t npad, cudaStream_t s) {
  k_split_df<<<(int)std::min<int64_t>((npad + 255) / 256, 2048), 256, 0, s>>>(x, hi, lo, n, npad); note_launch();
}

__device__ __forceinline__ void df_add4(DF& acc, const float4& a, const float4& bh, const float4& bl) {
  df_add_prod(acc, a.x, bh.x, bl.x);
  df_add_prod(acc, a.y, bh.y, bl.y);
  df_add_prod(acc, a.z, bh.z, bl.z);
  df_add_prod(acc, a.w, bh.w, bl.w);
}

__global__ void __launch_bounds__(256) k_rowdot_df(const float* __restrict__ J, int64_t ldJ, int64_t nrows,
                                                   const float* __restrict__ vh, const float* __restrict__ vl,
                                                   const double* __restrict__ w, double* __restrict__ t_out,
                                                   double* __restrict__ s_out, const int* __restrict__ done) {
  if (done && *done) return;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t nv = ldJ / 4;
  const float4* __restrict__ h4 = reinterpret_cast<const float4*>(vh);
  const float4* __restrict__ l4 = reinterpret_cast<const float4*>(vl);
  for (int64_t row = warp; row < nrows; row += nwarps) {
    const float4* __restrict__ jr = reinterpret_cast<const float4*>(J + row * ldJ);
    DF a0 = {0.f, 0.f}, a1 = {0.f, 0.f};
    int64_t k = lane;
    for (; k + 32 < nv; k += 64) {
      df_add4(a0, jr[k], h4[k], l4[k]);
      df_add4(a1, jr[k + 32], h4[k + 32], l4[k + 32]);
    }
    if (k < nv) df_add4(a0, jr[k], h4[k], l4[k]);
    const double tsum = wsum(((double)a0.hi + (double)a0.lo) + ((double)a1.hi + (double)a1.lo));
    if (lane == 0) {
      if (t_out) t_out[row] = tsum;
      if (s_out) s_out[row] = w ? w[row] * tsum : tsum;
    }
  }
}

void launch_rowdot_df(const float* J, int64_t ldJ, int64_t nrows, const float* vh, const float* vl, const double* w,
                      double* t_out, double* s_out, const int* done, cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>((nrows * 32 + 255) / 256, 152 * 16);
  k_rowdot_df<<<blocks, 256, 0, s>>>(J, ldJ, nrows, vh, vl, w, t_out, s_out, done); note_launch();
}

// The row scales s_n are split into FP32 pairs once per block, a chunk of rows at a time, into
// shared memory: splitting them in every thread put three FP64 operations per row and thread on
// GB300's narrow FP64 pipe, which then bounded the kernel instead of HBM.
__global__ void __launch_bounds__(256) k_coldot_df(const float* __restrict__ J, int64_t ldJ, int64_t nrows,
                                                   const double* __restrict__ sv, double* __restrict__ part,
                                                   int64_t rows_per_split, const int* __restrict__ done) {
  if (done && *done) return;
  constexpr int kChunk = 1024;
  __shared__ float2 ss[kChunk];
  const int64_t col = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  const bool active = col < ldJ;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_split;
  const int64_t r1 = min(nrows, r0 + rows_per_split);
  DF acc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  for (int64_t c0 = r0; c0 < r1; c0 += kChunk) {
    const int cn = (int)min((int64_t)kChunk, r1 - c0);
    __syncthreads();                                   // the previous chunk's scales are read
    for (int i = threadIdx.x; i < cn; i += blockDim.x) {
      float h, l;
      split_df(sv[c0 + i], h, l);
      ss[i] = make_float2(h, l);
    }
    __syncthreads();
    if (active) {
      const float* jc = J + c0 * ldJ + col;
      for (int i = 0; i < cn; ++i) {
        const float2 sc = ss[i];
        const float4 jv = *reinterpret_cast<const float4*>(jc + (int64_t)i * ldJ);
        df_add_prod(acc[0], jv.x, sc.x, sc.y);
        df_add_prod(acc[1], jv.y, sc.x, sc.y);
        df_add_prod(acc[2], jv.z, sc.x, sc.y);
        df_add_prod(acc[3], jv.w, sc.x, sc.y);
      }
    }
  }
  if (!active) return;
  double* pp = part + (int64_t)blockIdx.y * ldJ + col;
#pragma unroll
  for (int e = 0; e < 4; ++e) pp[e] = f32_to_f64(acc[e].hi) + f32_to_f64(acc[e].lo);
}

void launch_coldot_df(const float* J, int64_t ldJ, int64_t nrows, const double* s_vec, double* part, int nsplit,
                      const int* done, cudaStream_t st) {
  const int64_t rps = (nrows + nsplit - 1) / nsplit;
  dim3 grid((unsigned)((ldJ / 4 + 255) / 256), (unsigned)nsplit);
  k_coldot_df<<<grid, 256, 0, st>>>(J, ldJ, nrows, s_vec, part, rps, done); note_launch();
}

// y[j] = (accumulate ? y[j] : 0) + sum_split part[split][j] + mu v[j]   (mu from device or host)
__global__ void k_coldot_finish(const double* __restrict__ part, int nsplit, int64_t p, int64_t ld_part,
                                const double* __restrict__ v, double mu_h, const double* __restrict__ mu_d,
                                double* __restrict__ y, int accumulate, const int* __restrict__ done) {
  if (done && *done) return;
  const double mu = mu_d ? *mu_d : mu_h;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p; j += stride) {
    double s = accumulate ? y[j] : 0.0;
    for (int k = 0; k < nsplit; ++k) s += part[(int64_t)k * ld_part + j];
    if (v) s += mu * v[j];
    y[j] = s;
  }
}

void launch_coldot_finish(const double* part, int nsplit, int64_t p, int64_t ld_part, const double* v, double mu_h,
                          const double* mu_d, double* y, int accumulate, const int* done, cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>((p + 255) / 256, 1024);
  k_coldot_finish<<<blocks, 256, 0, s>>>(part, nsplit, p, ld_part, v, mu_h, mu_d, y, accumulate, done); note_launch();
}

// ---------------------------------------------------------------------------- vectors / PCG
__global__ void k_pcg_init(const double* __restrict__ g, double* __restrict__ x, double* __restrict__ r, int64_t n,
                           double* part, PcgScalars* sc) {
  __shared__ double red[32];
  double acc = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double gi = g[i];
    x[i] = 0.0;
    r[i] = gi;
    acc += gi * gi;
  }
  acc = block_sum(acc, red);
  double tot;
  if (last_block_total(acc, part, &sc->counter, &tot)) {
    sc->gn2 = tot;
    sc->cur_iter = 0;
    sc->iters = 0;
    sc->rn2 = tot;
    sc->done = (tot == 0.0 || sc->maxit <= 0) ? 1 : 0;
    if (!isfinite(tot)) {
      sc->status |= kStatNonFinite;
      sc->done = 1;
    }
  }
}

// p = z, rz = r . z
__global__ void k_pcg_first_dir(const double* __restrict__ r, const double* __restrict__ z, double* __restrict__ pv,
                                int64_t n, double* part, PcgScalars* sc) {
  __shared__ double red[32];
  double acc = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double zi = z[i];
    pv[i] = zi;
    acc += r[i] * zi;
  }
  acc = block_sum(acc, red);
  double tot;
  if (last_block_total(acc, part, &sc->counter, &tot)) sc->rz = tot;
}

// alpha = rz / (p . q)
__global__ void k_pcg_alpha(const double* __restrict__ pv, const double* __restrict__ q, int64_t n, double* part,
                            PcgScalars* sc) {
  if (sc->done) return;
  __shared__ double red[32];
  double acc = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) acc += pv[i] * q[i];
  acc = block_sum(acc, red);
  double tot;
  if (last_block_total(acc, part, &sc->counter, &tot)) {
    sc->pq = tot;
    if (!(tot > 0.0) || !isfinite(tot)) {
      sc->status |= isfinite(tot) ? kStatBreakdown : kStatNonFinite;
      sc->done = 1;
      sc->iters = sc->cur_iter;
    } else {
      sc->alpha = sc->rz / tot;
    }
  }
}

// x += alpha p, r -= alpha q, ||r||^2, convergence test
__global__ void k_pcg_update_xr(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ pv,
                                const double* __restrict__ q, int64_t n, double* part, PcgScalars* sc) {
  if (sc->done) return;
  __shared__ double red[32];
  const double alpha = sc->alpha;
  double acc = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    x[i] += alpha * pv[i];
    const double ri = r[i] - alpha * q[i];
    r[i] = ri;
    acc += ri * ri;
  }
  acc = block_sum(acc, red);
  double tot;
  if (last_block_total(acc, part, &sc->counter, &tot)) {
    const int it = sc->cur_iter + 1;
    sc->cur_iter = it;
    sc->iters = it;
    sc->rn2 = tot;
    if (!isfinite(tot)) {
      sc->status |= kStatNonFinite;
      sc->done = 1;
    } else if (tot <= sc->rtol2 * sc->gn2 || it >= sc->maxit) {
      sc->done = 1;
    }
  }
}

// rz_new = r . z, beta = rz_new / rz
__global__ void k_pcg_beta(const double* __restrict__ r, const double* __restrict__ z, int64_t n, double* part,
                           PcgScalars* sc) {
  if (sc->done) return;
  __shared__ double red[32];
  double acc = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) acc += r[i] * z[i];
  acc = block_sum(acc, red);
  double tot;
  if (last_block_total(acc, part, &sc->counter, &tot)) {
    sc->beta = tot / sc->rz;
    sc->rz = tot;
  }
}

// p = z + beta p
__global__ void k_pcg_update_p(double* __restrict__ pv, const double* __restrict__ z, int64_t n, PcgScalars* sc) {
  if (sc->done) return;
  const double beta = sc->beta;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) pv[i] = z[i] + beta * pv[i];
}

static int vec_blocks(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, kRedBlocks); }

void launch_pcg_init(const double* g, double* x, double* r, int64_t n, double* part, PcgScalars* sc,
                     cudaStream_t s) {
  k_pcg_init<<<vec_blocks(n), 256, 0, s>>>(g, x, r, n, part, sc); note_launch();
}
void launch_pcg_first_dir(const double* r, const double* z, double* pv, int64_t n, double* part, PcgScalars* sc,
                          cudaStream_t s) {
  k_pcg_first_dir<<<vec_blocks(n), 256, 0, s>>>(r, z, pv, n, part, sc); note_launch();
}
void launch_pcg_alpha(const double* pv, const double* q, int64_t n, double* part, PcgScalars* sc, cudaStream_t s) {
  k_pcg_alpha<<<vec_blocks(n), 256, 0, s>>>(pv, q, n, part, sc); note_launch();
}
void launch_pcg_update_xr(double* x, double* r, const double* pv, const double* q, int64_t n, double* part,
                          PcgScalars* sc, cudaStream_t s) {
  k_pcg_update_xr<<<vec_blocks(n), 256, 0, s>>>(x, r, pv, q, n, part, sc); note_launch();
}
void launch_pcg_beta(const double* r, const double* z, int64_t n, double* part, PcgScalars* sc, cudaStream_t s) {
  k_pcg_beta<<<vec_blocks(n), 256, 0, s>>>(r, z, n, part, sc); note_launch();
}
void launch_pcg_update_p(double* pv, const double* z, int64_t n, PcgScalars* sc, cudaStream_t s) {
  k_pcg_update_p<<<vec_blocks(n), 256, 0, s>>>(pv, z, n, sc); note_launch();
}

// y = x - alpha d  (Armijo trial point / final update)
__global__ void k_axpy_to(const double* __restrict__ x, const double* __restrict__ d, double alpha,
                          double* __restrict__ y, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) y[i] = x[i] - alpha * d[i];
}
void launch_axpy_to(const double* x, const double* d, double alpha, double* y, int64_t n, cudaStream_t s) {
  k_axpy_to<<<vec_blocks(n), 256, 0, s>>>(x, d, alpha, y, n); note_launch();
}

// dot product into *out (deterministic, two kernels: partials then ordered sum)
__global__ void k_dot_part(const double* __restrict__ a, const double* __restrict__ b, int64_t n, double* part) {
  __shared__ double red[32];
  double acc = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) acc += a[i] * b[i];
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}
void launch_dot(const double* a, const double* b, int64_t n, double* part, double* out, cudaStream_t s) {
  const int nb = vec_blocks(n);
  k_dot_part<<<nb, 256, 0, s>>>(a, b, n, part); note_launch();
  launch_sum_partials(part, nb, 1.0, out, s);
}

// ---------------------------------------------------------------------------- Nystrom preconditioner
// The scaled preconditioner maps the leading eigen-directions to (lam_ell + mu) / (lam_i + mu),
// which is ~ mu / lam_1 (1e-8 for the 5-D Poisson workload) and far below the FP32 unit
// roundoff, so its apply must be accurate to well below that: with FP32 arithmetic the computed
// P^{-1} v carries noise of ~1e-7 |v| and CG stalls.  FP32-stored U (float) is therefore applied
// with double-float (FP32 pair) accumulation: each FP32 product is split exactly with fmaf and
// summed by TwoSum (Knuth), which keeps ~2^-44 relative accuracy on the FP32 pipes instead of the
// scarce FP64 units.  FP64 U (double) uses FP64 arithmetic.
// w1[j] = sum_i U[i, j] v[i], four columns per block.
__global__ void __launch_bounds__(256) k_utv_f(const float* __restrict__ U, int64_t ld, int64_t p, int ell,
                                               const double* __restrict__ v, double* __restrict__ w1,
                                               const int* __restrict__ done) {
  if (done && *done) return;
  __shared__ double red[4][32];
  const int j0 = blockIdx.x * 4;
  DF acc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  for (int64_t i = threadIdx.x; i < p; i += blockDim.x) {
    float vh, vl;
    split_df(v[i], vh, vl);
#pragma unroll
    for (int c = 0; c < 4; ++c)
      if (j0 + c < ell) df_add_prod(acc[c], U[i + (int64_t)(j0 + c) * ld], vh, vl);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const double sv = wsum(f32_to_f64(acc[c].hi) + f32_to_f64(acc[c].lo));
    if (lane == 0) red[c][warp] = sv;
  }
  __syncthreads();
  if (threadIdx.x < 4 && j0 + (int)threadIdx.x < ell) {
    double sv = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sv += red[threadIdx.x][w];
    w1[j0 + threadIdx.x] = sv;
  }
}

__global__ void __launch_bounds__(256) k_utv_d(const double* __restrict__ U, int64_t ld, int64_t p, int ell,
                                               const double* __restrict__ v, double* __restrict__ w1,
                                               const int* __restrict__ done) {
  if (done && *done) return;
  __shared__ double red[4][32];
  const int j0 = blockIdx.x * 4;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t i = threadIdx.x; i < p; i += blockDim.x) {
    const double vi = v[i];
#pragma unroll
    for (int c = 0; c < 4; ++c)
      if (j0 + c < ell) acc[c] += U[i + (int64_t)(j0 + c) * ld] * vi;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const double sv = wsum(acc[c]);
    if (lane == 0) red[c][warp] = sv;
  }
  __syncthreads();
  if (threadIdx.x < 4 && j0 + (int)threadIdx.x < ell) {
    double sv = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sv += red[threadIdx.x][w];
    w1[j0 + threadIdx.x] = sv;
  }
}

// z[i] = v[i] + sum_j U[i, j] w2[j],  w2[j] = ((lam_ell + mu) / (lam_j + mu) - 1) w1[j]
__global__ void __launch_bounds__(256) k_precond_apply_f(const float* __restrict__ U, int64_t ld, int64_t p, int ell,
                                                         const double* __restrict__ lam, double mu_h,
                                                         const double* __restrict__ mu_d,
                                                         const double* __restrict__ w1, const double* __restrict__ v,
                                                         double* __restrict__ z, const int* __restrict__ done) {
  if (done && *done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* w2 = reinterpret_cast<float2*>(smem_raw);
  const double mu = mu_d ? *mu_d : mu_h;
  const double ln = lam[ell - 1] + mu;
  for (int j = threadIdx.x; j < ell; j += blockDim.x) {
    float h, l;
    split_df((ln / (lam[j] + mu) - 1.0) * w1[j], h, l);
    w2[j] = make_float2(h, l);
  }
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p; i += stride) {
    DF acc = {0.f, 0.f};
    for (int j = 0; j < ell; ++j) {
      const float2 ww = w2[j];
      df_add_prod(acc, U[i + (int64_t)j * ld], ww.x, ww.y);
    }
    z[i] = v[i] + (f32_to_f64(acc.hi) + f32_to_f64(acc.lo));
  }
}

__global__ void __launch_bounds__(256) k_precond_apply_d(const double* __restrict__ U, int64_t ld, int64_t p, int ell,
                                                         const double* __restrict__ lam, double mu_h,
                                                         const double* __restrict__ mu_d,
                                                         const double* __restrict__ w1, const double* __restrict__ v,
                                                         double* __restrict__ z, const int* __restrict__ done) {
  if (done && *done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* w2 = reinterpret_cast<double*>(smem_raw);
  const double mu = mu_d ? *mu_d : mu_h;
  const double ln = lam[ell - 1] + mu;
  for (int j = threadIdx.x; j < ell; j += blockDim.x) w2[j] = (ln / (lam[j] + mu) - 1.0) * w1[j];
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p; i += stride) {
    double a0 = 0.0, a1 = 0.0;
    int j = 0;
    for (; j + 1 < ell; j += 2) {
      a0 += U[i + (int64_t)j * ld] * w2[j];
      a1 += U[i + (int64_t)(j + 1) * ld] * w2[j + 1];
    }
    if (j < ell) a0 += U[i + (int64_t)j * ld] * w2[j];
    z[i] = v[i] + (a0 + a1);
  }
}

template <typename T>
void launch_precond(const T* U, int64_t ld, int64_t p, int ell, const double* lam, double mu_h, const double* mu_d,
                    const double* v, double* z, double* w1, const int* done, cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>((p + 255) / 256, 2048);
  if (sizeof(T) == 4) {
    k_utv_f<<<(ell + 3) / 4, 256, 0, s>>>((const float*)U, ld, p, ell, v, w1, done); note_launch();
    k_precond_apply_f<<<blocks, 256, ell * sizeof(float2), s>>>((const float*)U, ld, p, ell, lam, mu_h, mu_d, w1, v,
                                                                  z, done); note_launch();
  } else {
    k_utv_d<<<(ell + 3) / 4, 256, 0, s>>>((const double*)U, ld, p, ell, v, w1, done); note_launch();
    k_precond_apply_d<<<blocks, 256, ell * sizeof(double), s>>>((const double*)U, ld, p, ell, lam, mu_h, mu_d, w1, v,
                                                                   z, done); note_launch();
  }
}
template void launch_precond<float>(const float*, int64_t, int64_t, int, const double*, double, const double*,
                                    const double*, double*, double*, const int*, cudaStream_t);
template void launch_precond<double>(const double*, int64_t, int64_t, int, const double*, double, const double*,
                                     const double*, double*, double*, const int*, cudaStream_t);

// ---------------------------------------------------------------------------- Philox test matrix
// Philox4x32-10 (Salmon et al., SC'11): round (c0..c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2),
// hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)); key += (W0, W1) between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

__device__ __forceinline__ uint64_t bits52(uint32_t a, uint32_t b) {
  return ((((uint64_t)a) << 20) ^ (uint64_t)(b >> 12)) & ((1ull << 52) - 1ull);
}

__device__ __forceinline__ double uniform52(uint32_t a, uint32_t b) { return ((double)bits52(a, b) + 0.5) * 0x1p-52; }

// N 2^e rounded to FP32 (nearest, ties to even) for 0 < N < 2^62, by integer operations (GB300
// runs integer-to-float conversions of 64-bit values through its narrow FP64 pipe).
__device__ __forceinline__ float u64_scaled_to_f32(uint64_t N, int e) {
  const int top = 63 - __clzll((long long)N);              // N in [2^top, 2^(top+1))
  uint32_t mant;
  if (top > 23) {
    const int sh = top - 23;
    const uint64_t q = N >> sh, rem = N & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    mant = (uint32_t)q + ((rem > half || (rem == half && (q & 1ull))) ? 1u : 0u);
  } else {
    mant = (uint32_t)(N << (23 - top));
  }
  int ex = top + e;
  if (mant >> 24) {                                        // rounded up to 2^24
    mant >>= 1;
    ++ex;
  }
  return __uint_as_float((uint32_t)(ex + 127) << 23 | (mant & 0x7fffffu));
}

// One Box-Muller pair in FP32 arithmetic for an FP32 test matrix: u1 = (m1 + 1/2) 2^-52 and
// u2 = (m2 + 1/2) 2^-52 as above; log u1 from the exact complement for u1 >= 1/2 (log1p of -(1 - u1),
// so that u1 near 1 keeps its low bits), 2 pi u2 reduced exactly to a quadrant (the top two bits
// of m2) plus (pi / 2) f, f in (0, 1), and f above 1/2 to its exact complement (sine and cosine
// swapped), with FP32 sinpi / cospi of an argument in (0, 1/4].  Each value is within a few units
// of FP32 rounding, relative to the pair's radius, of the FP64 pair.
__device__ __forceinline__ void box_muller_f32(uint64_t m1, uint64_t m2, float& g0, float& g1) {
  float L;
  if (m1 >> 51) L = log1pf(-u64_scaled_to_f32(2ull * ((1ull << 52) - 1ull - m1) + 1ull, -53));
  else L = logf(u64_scaled_to_f32(2ull * m1 + 1ull, -53));
  const float rr = sqrtf(-2.f * L);
  const int q = (int)(m2 >> 50);
  const uint64_t F = 2ull * (m2 & ((1ull << 50) - 1ull)) + 1ull;   // f = F 2^-51
  float sn, cs;                                            // sin, cos of (pi / 2) f
  if (F >> 50) {                                           // f > 1/2: from the exact complement 1 - f
    sincospif(0.5f * u64_scaled_to_f32((1ull << 51) - F, -51), &cs, &sn);
  } else {
    sincospif(0.5f * u64_scaled_to_f32(F, -51), &sn, &cs);
  }
  float c = cs, s = sn;                                    // cos, sin of q pi / 2 + (pi / 2) f
  if (q == 1) { c = -sn; s = cs; }
  else if (q == 2) { c = -cs; s = -sn; }
  else if (q == 3) { c = sn; s = -cs; }
  g0 = rr * c;
  g1 = rr * s;
}

// Omega[i + j*ld] for i < p (rows 2m, 2m+1 from counter (m, j, step_lo, step_hi), key (seed_lo, seed_hi)).
template <typename T>
__global__ void k_philox_omega(T* __restrict__ Om, int64_t ld, int64_t p, int ell, uint64_t seed, uint64_t step) {
  const int64_t npairs = (p + 1) / 2;
  const int64_t total = npairs * ell;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
    const int j = (int)(t / npairs);
    const int64_t m = t - (int64_t)j * npairs;
    const uint4 x = philox4x32_10(make_uint4((uint32_t)m, (uint32_t)j, (uint32_t)step, (uint32_t)(step >> 32)),
                                  (uint32_t)seed, (uint32_t)(seed >> 32));
    T* col = Om + (int64_t)j * ld;
    if constexpr (sizeof(T) == 4) {
      float g0, g1;
      box_muller_f32(bits52(x.x, x.y), bits52(x.z, x.w), g0, g1);
      col[2 * m] = g0;
      if (2 * m + 1 < p) col[2 * m + 1] = g1;
    } else {
      const double u1 = uniform52(x.x, x.y), u2 = uniform52(x.z, x.w);
      const double rr = sqrt(-2.0 * log(u1));
      double sn, cs;
      sincospi(2.0 * u2, &sn, &cs);
      col[2 * m] = (T)(rr * cs);
      if (2 * m + 1 < p) col[2 * m + 1] = (T)(rr * sn);
    }
  }
}

template <typename T>
void launch_philox_omega(T* Om, int64_t ld, int64_t p, int ell, uint64_t seed, uint64_t step, cudaStream_t s) {
  const int64_t total = (p + 1) / 2 * ell;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 8192);
  k_philox_omega<T><<<blocks, 256, 0, s>>>(Om, ld, p, ell, seed, step); note_launch();
}
template void launch_philox_omega<float>(float*, int64_t, int64_t, int, uint64_t, uint64_t, cudaStream_t);
template void launch_philox_omega<double>(double*, int64_t, int64_t, int, uint64_t, uint64_t, cudaStream_t);

// ---------------------------------------------------------------------------- sampling test matrix
// diag(G)_j = sum_n w_n J[n, j]^2 (Eq. gram_diagonal) over the nrows rows of J (row n at J + n ldJ,
// weight w[n]), FP64 accumulation; rows split z (rows_per_split each) into part[z * ldp + j]
// (added to it when accumulate).  Threads of a warp take consecutive j: coalesced rows of J.
template <typename T>
__global__ void k_gram_diag(const T* __restrict__ J, int64_t ldJ, int64_t nrows, int64_t p, const double* __restrict__ w,
                            int64_t rows_per_split, double* __restrict__ part, int64_t ldp, int accumulate) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= p) return;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_split, r1 = min(nrows, r0 + rows_per_split);
  double s = 0.0;
  for (int64_t r = r0; r < r1; ++r) {
    const double x = (double)J[r * ldJ + j];
    s += w[r] * x * x;
  }
  double* o = part + (int64_t)blockIdx.y * ldp + j;
  *o = accumulate ? *o + s : s;
}
template <typename T>
int launch_gram_diag(const T* J, int64_t ldJ, int64_t nrows, int64_t p, const double* w, double* part, int64_t ldp,
                     int max_splits, int accumulate, cudaStream_t s) {
  const int64_t rps = std::max<int64_t>(64, (nrows + max_splits - 1) / max_splits);
  const int nz = (int)std::max<int64_t>(1, (nrows + rps - 1) / rps);
  dim3 grid((unsigned)((p + 255) / 256), (unsigned)nz);
  k_gram_diag<T><<<grid, 256, 0, s>>>(J, ldJ, nrows, p, w, rps, part, ldp, accumulate); note_launch();
  return nz;
}
template int launch_gram_diag<float>(const float*, int64_t, int64_t, int64_t, const double*, double*, int64_t, int,
                                     int, cudaStream_t);
template int launch_gram_diag<double>(const double*, int64_t, int64_t, int64_t, const double*, double*, int64_t, int,
                                      int, cudaStream_t);

// Keys of an exponential race (Efraimidis & Spirakis, 2006): the ell smallest of
// E_j = -ln(u_j) / d_j, u_j uniform from the Philox counter (j, 2^32 - 1, step_lo, step_hi) and key
// (seed_lo, seed_hi), are a sample of ell distinct indices drawn one after another with
// probabilities proportional to d among those not yet drawn.  d_j <= 0 (or not finite) never
// wins (key +inf).  Keys are stored as the bits of the non-negative double, which order like it.
__global__ void k_sample_keys(const double* __restrict__ d, int64_t p, uint64_t seed, uint64_t step,
                              unsigned long long* __restrict__ keys) {
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p; j += st) {
    const uint4 x = philox4x32_10(make_uint4((uint32_t)j, 0xFFFFFFFFu, (uint32_t)step, (uint32_t)(step >> 32)),
                                  (uint32_t)seed, (uint32_t)(seed >> 32));
    const double dj = d[j];
    const double e = (dj > 0.0 && isfinite(dj)) ? -log(uniform52(x.x, x.y)) / dj : CUDART_INF;
    keys[j] = (unsigned long long)__double_as_longlong(e);
  }
}

// number of keys <= t over the block (every thread gets it); s: 33 shared words
__device__ long long block_count_le(const unsigned long long* __restrict__ keys, int64_t p, unsigned long long t,
                                   long long* s) {
  long long c = 0;
  for (int64_t j = threadIdx.x; j < p; j += blockDim.x) c += keys[j] <= t ? 1 : 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t2 = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t2 += s[w];
    s[32] = t2;
  }
  __syncthreads();
  const long long r = s[32];
  __syncthreads();
  return r;
}

// exclusive prefix sum of v over the threads of the block in thread order; s: 33 shared words
__device__ long long block_exclusive_scan(long long v, long long* s) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s[warp] = x;
  __syncthreads();
  if (warp == 0) {
    long long w = lane < nw ? s[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    s[lane] = w;
  }
  __syncthreads();
  const long long r = (warp > 0 ? s[warp - 1] : 0) + x - v;
  __syncthreads();
  return r;
}

// The ell smallest keys (ties to the smaller index), written to idx in increasing index order:
// one block finds the ell-th smallest key T by bisection on its bits, then takes every key below
// T and the first ell - #(below) keys equal to T.  Fewer than ell finite keys: status bit
// kStatSample, idx untouched.
__global__ void __launch_bounds__(1024) k_sample_select(const unsigned long long* __restrict__ keys, int64_t p, int ell,
                                                        int* __restrict__ idx, int* __restrict__ status) {
  __shared__ long long s[33];
  const unsigned long long kInf = 0x7FF0000000000000ull;
  if (block_count_le(keys, p, kInf - 1, s) < ell) {
    if (threadIdx.x == 0) atomicOr(status, kStatSample);
    return;
  }
  unsigned long long lo = 0, hi = kInf - 1;
  while (lo < hi) {
    const unsigned long long mid = lo + (hi - lo) / 2;
    if (block_count_le(keys, p, mid, s) >= ell) hi = mid;
    else lo = mid + 1;
  }
  const unsigned long long T = lo;
  const long long need = ell - (T > 0 ? block_count_le(keys, p, T - 1, s) : 0);
  const int64_t chunk = (p + blockDim.x - 1) / blockDim.x;
  const int64_t j0 = min(p, (int64_t)threadIdx.x * chunk), j1 = min(p, j0 + chunk);
  long long eq = 0;
  for (int64_t j = j0; j < j1; ++j) eq += keys[j] == T ? 1 : 0;
  const long long eq_base = block_exclusive_scan(eq, s);
  long long sel = 0, e = eq_base;
  for (int64_t j = j0; j < j1; ++j) {
    const unsigned long long k = keys[j];
    if (k < T) ++sel;
    else if (k == T) sel += (e++ < need) ? 1 : 0;
  }
  long long o = block_exclusive_scan(sel, s);
  e = eq_base;
  for (int64_t j = j0; j < j1; ++j) {
    const unsigned long long k = keys[j];
    bool take = k < T;
    if (k == T) take = e++ < need;
    if (take) idx[o++] = (int)j;
  }
}

void launch_sample_indices(const double* d, int64_t p, int ell, uint64_t seed, uint64_t step,
                           unsigned long long* keys, int* idx, int* status, cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>((p + 255) / 256, 1024);
  k_sample_keys<<<blocks, 256, 0, s>>>(d, p, seed, step, keys); note_launch();
  k_sample_select<<<1, 1024, 0, s>>>(keys, p, ell, idx, status); note_launch();
}

// Omega[idx_k + k ld] = 1 (the rest already zero): the column-selection test matrix
template <typename T>
__global__ void k_selection_omega(T* __restrict__ Om, int64_t ld, const int* __restrict__ idx, int ell) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < ell) Om[(int64_t)idx[k] + (int64_t)k * ld] = T(1);
}
template <typename T>
void launch_selection_omega(T* Om, int64_t ld, const int* idx, int ell, cudaStream_t s) {
  k_selection_omega<T><<<(ell + 255) / 256, 256, 0, s>>>(Om, ld, idx, ell); note_launch();
}
template void launch_selection_omega<float>(float*, int64_t, const int*, int, cudaStream_t);
template void launch_selection_omega<double>(double*, int64_t, const int*, int, cudaStream_t);

// Zw[n ell + k] = w_n J[n, idx_k] (N x ell, row-major): diag(w) J Omega for a column-selection Omega
template <typename T, typename TO>
__global__ void k_gather_cols(const T* __restrict__ J, int64_t ldJ, int64_t N, const int* __restrict__ idx, int ell,
                              const double* __restrict__ w, TO* __restrict__ Zw) {
  const int64_t total = N * ell;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += st) {
    const int64_t n = e / ell;
    const int k = (int)(e - n * ell);
    Zw[e] = (TO)(w[n] * (double)J[n * ldJ + idx[k]]);
  }
}
template <typename T, typename TO>
void launch_gather_cols(const T* J, int64_t ldJ, int64_t N, const int* idx, int ell, const double* w, TO* Zw,
                        cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>((N * ell + 255) / 256, 8192);
  k_gather_cols<T, TO><<<blocks, 256, 0, s>>>(J, ldJ, N, idx, ell, w, Zw); note_launch();
}
template void launch_gather_cols<float, double>(const float*, int64_t, int64_t, const int*, int, const double*,
                                                double*, cudaStream_t);
template void launch_gather_cols<float, float>(const float*, int64_t, int64_t, const int*, int, const double*, float*,
                                               cudaStream_t);
template void launch_gather_cols<double, double>(const double*, int64_t, int64_t, const int*, int, const double*,
                                                 double*, cudaStream_t);

// ---------------------------------------------------------------------------- RPCholesky (App. B, Alg. 5)
// Gaussian vector v (p) from the test-matrix generator with column word `word` (rows 2m, 2m+1 from
// counter (m, word, step_lo, step_hi)): the power method's start vector uses word 2^32 - 2.
__global__ void k_philox_column(double* __restrict__ v, int64_t p, uint32_t word, uint64_t seed, uint64_t step) {
  const int64_t npairs = (p + 1) / 2;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < npairs; m += st) {
    const uint4 x = philox4x32_10(make_uint4((uint32_t)m, word, (uint32_t)step, (uint32_t)(step >> 32)),
                                  (uint32_t)seed, (uint32_t)(seed >> 32));
    const double u1 = uniform52(x.x, x.y), u2 = uniform52(x.z, x.w);
    const double rr = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    v[2 * m] = rr * cs;
    if (2 * m + 1 < p) v[2 * m + 1] = rr * sn;
  }
}
void launch_philox_column(double* v, int64_t p, uint32_t word, uint64_t seed, uint64_t step, cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>(((p + 1) / 2 + 255) / 256, 1024);
  k_philox_column<<<blocks, 256, 0, s>>>(v, p, word, seed, step); note_launch();
}

// dst = src / sqrt(*ss)
__global__ void k_scale_rsqrt(const double* __restrict__ src, const double* __restrict__ ss, double* __restrict__ dst,
                              int64_t n) {
  const double f = 1.0 / sqrt(*ss);
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += st) dst[i] = src[i] * f;
}
void launch_scale_rsqrt(const double* src, const double* ss, double* dst, int64_t n, cudaStream_t s) {
  k_scale_rsqrt<<<(int)std::min<int64_t>((n + 255) / 256, 1024), 256, 0, s>>>(src, ss, dst, n); note_launch();
}

// Round rnd of block RPCholesky: sample k (block k) is the winner of the race
// argmin_j -ln(u_jk) / d_j, u_jk from the counter (j, 2^30 + rnd b + k, step_lo, step_hi); ties to
// the smaller j.  piv[k] = -1 when every d_j <= 0.
__global__ void __launch_bounds__(256) k_rpchol_pivots(const double* __restrict__ d, int64_t p, int b, int rnd,
                                                       uint64_t seed, uint64_t step, int* __restrict__ piv) {
  __shared__ unsigned long long sk[256];
  __shared__ long long sj[256];
  const int k = blockIdx.x;
  const uint32_t word = (1u << 30) + (uint32_t)(rnd * b + k);
  unsigned long long best = ~0ull;
  long long bj = -1;
  for (int64_t j = threadIdx.x; j < p; j += blockDim.x) {
    const double dj = d[j];
    if (!(dj > 0.0) || !isfinite(dj)) continue;
    const uint4 x = philox4x32_10(make_uint4((uint32_t)j, word, (uint32_t)step, (uint32_t)(step >> 32)),
                                  (uint32_t)seed, (uint32_t)(seed >> 32));
    const unsigned long long key = (unsigned long long)__double_as_longlong(-log(uniform52(x.x, x.y)) / dj);
    if (key < best) {                       // j increases: the first of equal keys is kept
      best = key;
      bj = j;
    }
  }
  sk[threadIdx.x] = best;
  sj[threadIdx.x] = bj;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      const unsigned long long k2 = sk[threadIdx.x + o];
      const long long j2 = sj[threadIdx.x + o];
      if (j2 >= 0 && (sj[threadIdx.x] < 0 || k2 < sk[threadIdx.x] || (k2 == sk[threadIdx.x] && j2 < sj[threadIdx.x]))) {
        sk[threadIdx.x] = k2;
        sj[threadIdx.x] = j2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) piv[k] = (int)sj[0];
}

// The b pivots of a round made unique and increasing (piv < 0 dropped); count written to *nsel.
__global__ void k_unique_pivots(const int* __restrict__ piv, int b, int* __restrict__ sel, int* __restrict__ nsel) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int n = 0;
  for (int k = 0; k < b; ++k) {
    const int v = piv[k];
    if (v < 0) continue;
    int pos = n;
    bool dup = false;
    for (int i = 0; i < n; ++i) {
      if (sel[i] == v) { dup = true; break; }
      if (sel[i] > v) { pos = i; break; }
    }
    if (dup) continue;
    for (int i = n; i > pos; --i) sel[i] = sel[i - 1];
    sel[pos] = v;
    ++n;
  }
  *nsel = n;
}

void launch_rpchol_pivots(const double* d, int64_t p, int b, int rnd, uint64_t seed, uint64_t step, int* piv,
                          int* sel, int* nsel, cudaStream_t s) {
  k_rpchol_pivots<<<b, 256, 0, s>>>(d, p, b, rnd, seed, step, piv); note_launch();
  k_unique_pivots<<<1, 32, 0, s>>>(piv, b, sel, nsel); note_launch();
}

// Fs[k + n r] = -F[sel_n, k] (r x nsel, column-major): minus the pivot rows of F, transposed
__global__ void k_gather_rows_neg(const double* __restrict__ F, int64_t ld, const int* __restrict__ sel, int nsel, int r,
                                  double* __restrict__ Fs) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= r * nsel) return;
  const int k = e % r, n = e / r;
  Fs[e] = -F[(int64_t)sel[n] + (int64_t)k * ld];
}
void launch_gather_rows_neg(const double* F, int64_t ld, const int* sel, int nsel, int r, double* Fs, cudaStream_t s) {
  if (r <= 0 || nsel <= 0) return;
  k_gather_rows_neg<<<(r * nsel + 255) / 256, 256, 0, s>>>(F, ld, sel, nsel, r, Fs); note_launch();
}

// M = sym(C[sel, :]) (nsel x nsel, column-major) of the p x nsel residual block C (ld)
__global__ void k_pivot_block(const double* __restrict__ C, int64_t ld, const int* __restrict__ sel, int nsel,
                              double* __restrict__ M) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nsel * nsel) return;
  const int a = e % nsel, c = e / nsel;
  M[e] = 0.5 * (C[(int64_t)sel[a] + (int64_t)c * ld] + C[(int64_t)sel[c] + (int64_t)a * ld]);
}
void launch_pivot_block(const double* C, int64_t ld, const int* sel, int nsel, double* M, cudaStream_t s) {
  k_pivot_block<<<(nsel * nsel + 255) / 256, 256, 0, s>>>(C, ld, sel, nsel, M); note_launch();
}

// d_j <- max(0, d_j - sum_k F_new[j, k]^2), 0 on the pivots; block partial sums of the new d in part
__global__ void k_rpchol_diag(double* __restrict__ d, const double* __restrict__ Fn, int64_t ld, int64_t p, int nsel,
                              const int* __restrict__ sel, double* __restrict__ part) {
  __shared__ double red[32];
  double acc = 0.0;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < p; j += st) {
    double s2 = 0.0;
    bool piv = false;
    for (int k = 0; k < nsel; ++k) {
      const double f = Fn[j + (int64_t)k * ld];
      s2 += f * f;
      piv |= sel[k] == (int)j;
    }
    const double v = piv ? 0.0 : fmax(0.0, d[j] - s2);
    d[j] = v;
    acc += v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}
int launch_rpchol_diag(double* d, const double* Fn, int64_t ld, int64_t p, int nsel, const int* sel, double* part,
                       cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>((p + 255) / 256, 256);
  k_rpchol_diag<<<blocks, 256, 0, s>>>(d, Fn, ld, p, nsel, sel, part); note_launch();
  return blocks;
}

// lam_k = sigma_k^2 of F (descending) where sigma_k^2 > 2^-40 sigma_1^2, else 0 (that direction is
// left to the mu part of P); inv_sigma_k = 1 / sigma_k for the kept ones, 0 otherwise; lam[r] = 0.
__global__ void k_rpchol_lambda(const double* __restrict__ sig2, int r, double* __restrict__ lam,
                                double* __restrict__ inv_sigma) {
  const double top = r > 0 ? sig2[0] : 0.0;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= r; k += gridDim.x * blockDim.x) {
    const double s2 = k < r ? sig2[k] : 0.0;
    const bool keep = s2 > 0x1p-40 * top && s2 > 0.0;
    lam[k] = keep ? s2 : 0.0;
    inv_sigma[k] = keep ? 1.0 / sqrt(s2) : 0.0;
  }
}
void launch_rpchol_lambda(const double* sig2, int r, double* lam, double* inv_sigma, cudaStream_t s) {
  k_rpchol_lambda<<<(r + 1 + 255) / 256, 256, 0, s>>>(sig2, r, lam, inv_sigma); note_launch();
}

// ---------------------------------------------------------------------------- NGD full (Alg. 2)
// Z[n ld + j] = w_n J[n ld + j] in FP64 (N x ld row-major, the padding columns stay zero)
template <typename T>
__global__ void k_scale_rows_f64(const T* __restrict__ J, int64_t ld, int64_t N, const double* __restrict__ w,
                                 double* __restrict__ Z) {
  const int64_t total = N * ld;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += st)
    Z[e] = w[e / ld] * (double)J[e];
}
template <typename T>
void launch_scale_rows_f64(const T* J, int64_t ld, int64_t N, const double* w, double* Z, cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>((N * ld + 255) / 256, 8192);
  k_scale_rows_f64<T><<<blocks, 256, 0, s>>>(J, ld, N, w, Z); note_launch();
}
template void launch_scale_rows_f64<float>(const float*, int64_t, int64_t, const double*, double*, cudaStream_t);
template void launch_scale_rows_f64<double>(const double*, int64_t, int64_t, const double*, double*, cudaStream_t);

// A[i + i ld] += *shift
__global__ void k_add_diag_dev(double* __restrict__ A, int64_t n, int64_t ld, const double* __restrict__ shift) {
  const double sh = *shift;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += st) A[i + i * ld] += sh;
}
void launch_add_diag_dev(double* A, int64_t n, int64_t ld, const double* shift, cudaStream_t s) {
  k_add_diag_dev<<<(int)std::min<int64_t>((n + 255) / 256, 1024), 256, 0, s>>>(A, n, ld, shift); note_launch();
}

// A's strict upper triangle from its lower one (n x n, column-major, ld)
__global__ void k_lower_to_upper(double* __restrict__ A, int64_t n, int64_t ld) {
  const int64_t total = n * n;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += st) {
    const int64_t i = e % n, j = e / n;
    if (i < j) A[i + j * ld] = A[j + i * ld];
  }
}
void launch_lower_to_upper(double* A, int64_t n, int64_t ld, cudaStream_t s) {
  k_lower_to_upper<<<(int)std::min<int64_t>((n * n + 255) / 256, 8192), 256, 0, s>>>(A, n, ld); note_launch();
}

// T[k + j nb] = -X[j + k ld] (nb x m): the negated, transposed panel for the trailing update's GEMM
__global__ void k_neg_copy(const double* __restrict__ X, int64_t ld, int64_t m, int nb, double* __restrict__ T) {
  const int64_t total = m * nb;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += st) {
    const int64_t k = e % nb, j = e / nb;
    T[e] = -X[j + k * ld];
  }
}

// Right-looking blocked Cholesky A = L L^T for large n (A n x n, column-major, leading dimension
// lda; L into the lower triangle, the strict upper triangle left as it was): diagonal blocks of 256
// by the cooperative k_cholesky (through the contiguous scratch D), the panel below them by
// launch_trsm_lt, the trailing matrix by the double-float GEMM on its lower triangle
// (A22 -= P P^T).  A non-positive-definite pivot block sets kStatNotSpd in *status; the later
// blocks then compute on meaningless but finite-or-NaN values and write nothing outside A.
// D: 256 x 256 doubles; W: 256 x 256 doubles; T: 256 x (n - 256) doubles.  An even lda keeps
// the GEMM on its vectorised path.
cudaError_t launch_cholesky_blocked(double* A, int64_t n, int64_t lda, int* status, double* D, double* W, double* T,
                                    cudaStream_t s, OzSketch* oz, long long wait_cycles) {
  constexpr int nb = 256;
  for (int64_t k0 = 0; k0 < n; k0 += nb) {
    const int bs = (int)std::min<int64_t>(nb, n - k0);
    double* Akk = A + k0 + k0 * lda;
    cudaError_t e = cudaMemcpy2DAsync(D, (size_t)bs * 8, Akk, (size_t)lda * 8, (size_t)bs * 8, bs,
                                      cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    e = launch_cholesky(D, bs, status, s);                  // lower triangle of D; its upper one kept
    if (e != cudaSuccess) return e;
    e = cudaMemcpy2DAsync(Akk, (size_t)lda * 8, D, (size_t)bs * 8, (size_t)bs * 8, bs, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    const int64_t m = n - k0 - bs;
    if (m <= 0) break;
    double* P = Akk + bs;                                   // rows k0 + bs .., columns k0 .. k0 + bs
    launch_trsm_lt<double>(P, lda, m, bs, D, W, s);         // P <- P L_kk^{-T}
    if (oz) {                                               // lower(A22) -= P P^T on the tensor cores
      const char* why = nullptr;
      e = oz_syrk_sub(oz, P, lda, m, bs, Akk + bs + bs * lda, lda, &why, s, status, wait_cycles);
      if (e != cudaSuccess) return e;
      if (!why) continue;
    }
    k_neg_copy<<<(int)std::min<int64_t>((m * bs + 255) / 256, 8192), 256, 0, s>>>(P, lda, m, bs, T); note_launch();
    GemmDfArgs<double, double> g;                           // lower(A22) += lower(P (-P^T))
    g.M = m; g.N = m; g.K = bs;
    g.A = P; g.sam = 1; g.sak = lda;
    g.B = T; g.sbk = 1; g.sbn = bs;                         // B[k][j] = T[k + j bs] = -P[j, k]
    g.out64 = Akk + bs + bs * lda; g.scm = 1; g.scn = lda;
    g.accumulate = 1;
    g.lower = 1;
    launch_gemm_df<double, double>(g, s);
  }
  return cudaGetLastError();
}

// dg = diag(A) (before the shift and the in-place Cholesky, which only writes the lower triangle)
__global__ void k_copy_diag(const double* __restrict__ A, int64_t n, int64_t ld, double* __restrict__ dg) {
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += st) dg[i] = A[i + i * ld];
}
void launch_copy_diag(const double* A, int64_t n, int64_t ld, double* dg, cudaStream_t s) {
  k_copy_diag<<<(int)std::min<int64_t>((n + 255) / 256, 1024), 256, 0, s>>>(A, n, ld, dg); note_launch();
}
// A's lower triangle again from its untouched strict upper triangle, diagonal dg + *shift
__global__ void k_restore_lower(double* __restrict__ A, int64_t n, int64_t ld, const double* __restrict__ dg,
                                const double* __restrict__ shift) {
  const double sh = *shift;
  const int64_t total = n * n;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += st) {
    const int64_t i = e % n, j = e / n;                    // A[i + j ld], lower when i >= j
    if (i > j) A[i + j * ld] = A[j + i * ld];
    else if (i == j) A[i + j * ld] = dg[i] + sh;
  }
}
void launch_restore_lower(double* A, int64_t n, int64_t ld, const double* dg, const double* shift, cudaStream_t s) {
  k_restore_lower<<<(int)std::min<int64_t>((n * n + 255) / 256, 8192), 256, 0, s>>>(A, n, ld, dg, shift);
  note_launch();
}
__global__ void k_scale_scalar(double* __restrict__ x, double f) { *x *= f; }
void launch_scale_scalar(double* x, double f, cudaStream_t s) {
  k_scale_scalar<<<1, 1, 0, s>>>(x, f); note_launch();
}

// x = (L L^T)^{-1} b for the lower Cholesky factor L (n x n, column-major, leading dimension ld):
// forward then backward substitution by blocks of kCsB rows in one cooperative launch, one grid
// barrier per block.  Block 0 owns the sequential part: its warp 0 solves each diagonal block from
// shared memory (lanes hold two rows each), the block staged there while the other blocks wait at
// the previous barrier, its strictly lower entries already divided by the pivot that multiplies
// them (column pivots forward, row pivots backward), so that the dependent chain is one shuffle
// and the FMAs of the rows still open per column, and the solved piece is scaled by the
// reciprocal pivots at the end.  After the barrier every block reads the solved piece, and the
// rows still to be updated are: the next diagonal block's rows by block 0 itself (look-ahead), so
// that block 0 can solve it at once, and the rest by the other blocks.  A row's earlier updates by
// other blocks lie at least one barrier back.  Each row's kCsB-term update is split over four
// threads (a quarter of the columns each) and combined in shared memory, so that every warp-wide
// FP64 instruction carries 32 rows: GB300's FP64 pipe retires about two FMAs per clock and SM.
// All arithmetic FP64.  y: scratch of n; gridDim.x >= 2, blockDim.x = kCsT.
constexpr int kCsB = 64;           // rows per diagonal block
constexpr int kCsLd = kCsB + 1;    // padded leading dimension of the staged diagonal block
constexpr int kCsT = 256;          // threads per block: kCsB rows x 4 quarters of the columns
static_assert(kCsT == 4 * kCsB, "one row per four threads");

// block 0: diagonal block of L at (k0, k0), bs x bs, into Ls (column-major, ld kCsLd) with only its
// strictly lower entries kept, each divided by its column's pivot (fwd) or its row's pivot (bwd);
// 1 / L_jj into rd.
__device__ __forceinline__ void cs_stage_diag(const double* __restrict__ L, int64_t ld, int k0, int bs, bool fwd,
                                              double* __restrict__ Ls, double* __restrict__ rd) {
  if ((int)threadIdx.x < bs) rd[threadIdx.x] = 1.0 / L[(int64_t)(k0 + threadIdx.x) * (ld + 1)];
  __syncthreads();
  for (int e = threadIdx.x; e < kCsB * kCsB; e += blockDim.x) {
    const int r = e % kCsB, c = e / kCsB;
    Ls[c * kCsLd + r] = (r < bs && c < r) ? L[(int64_t)(k0 + r) + (int64_t)(k0 + c) * ld] * rd[fwd ? c : r] : 0.0;
  }
}

// y[i] -= sum_{j < bs} L(i, j) blk[j] for the rows i = row(r), r = r0 + (tid mod kCsB),
// r0 + kCsB G', ... < r1, where L(i, j) = L[i + (k0 + j) ld] (fwd) or L[k0 + j + i ld] (bwd):
// four threads per row, a quarter of the j each.  Every thread of the block calls it.
__device__ __forceinline__ void cs_update_rows(const double* __restrict__ L, int64_t ld, int k0, int bs, bool fwd,
                                               int64_t r0, int64_t r1, int64_t rstride, int64_t base, int64_t dir,
                                               const double* __restrict__ blk, double* __restrict__ red,
                                               double* __restrict__ v) {
  const int rr = threadIdx.x % kCsB, q = threadIdx.x / kCsB;
  constexpr int kQ = kCsB / 4;
  for (int64_t r = r0; r < r1; r += rstride) {              // r0, r1, rstride the same in the whole block
    const int64_t rt = r + rr;
    const bool on = rt < r1;
    const int64_t i = base + dir * rt;
    double s0 = 0.0, s1 = 0.0;
    if (on) {
#pragma unroll
      for (int t = 0; t < kQ; t += 2) {
        const int j = q * kQ + t;
        const double l0 = j < bs ? (fwd ? L[i + (int64_t)(k0 + j) * ld] : L[k0 + j + i * ld]) : 0.0;
        const double l1 = j + 1 < bs ? (fwd ? L[i + (int64_t)(k0 + j + 1) * ld] : L[k0 + j + 1 + i * ld]) : 0.0;
        s0 = fma(l0, blk[j], s0);
        s1 = fma(l1, blk[j + 1], s1);
      }
    }
    red[q * kCsB + rr] = s0 + s1;
    __syncthreads();
    if (q == 0 && on) v[i] = __ldcg(v + i) - ((red[rr] + red[kCsB + rr]) + (red[2 * kCsB + rr] + red[3 * kCsB + rr]));
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kCsT) k_chol_solve(const double* __restrict__ L, int n, int64_t ld,
                                                    const double* __restrict__ b,
                                                    double* __restrict__ x, double* __restrict__ y) {
  cg::grid_group grid = cg::this_grid();
  __shared__ double Ls[kCsB * kCsLd];
  __shared__ double rd[kCsB];
  __shared__ double blk[kCsB];
  __shared__ double red[4 * kCsB];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, gthreads = (int64_t)gridDim.x * blockDim.x;
  const bool b0 = blockIdx.x == 0;
  // rows of the other blocks: kCsB per block and pass, passes over the G - 1 blocks
  const int64_t orow0 = (int64_t)(blockIdx.x - 1) * kCsB, ostride = (int64_t)(gridDim.x - 1) * kCsB;
  for (int64_t i = gtid; i < n; i += gthreads) y[i] = b[i];
  if (b0 && n > 0) cs_stage_diag(L, ld, 0, min(kCsB, n), true, Ls, rd);
  grid.sync();
  for (int k0 = 0; k0 < n; k0 += kCsB) {                    // L y = b
    const int bs = min(kCsB, n - k0);
    if (b0) {
      __syncthreads();                                      // look-ahead rows and the staged block
      if (warp == 0) {
        double ya = lane < bs ? __ldcg(y + k0 + lane) : 0.0;
        double yb = lane + 32 < bs ? __ldcg(y + k0 + 32 + lane) : 0.0;
        for (int j = 0; j < bs; ++j) {                      // unscaled: pivots applied at the end
          const double yj = __shfl_sync(0xffffffffu, j < 32 ? ya : yb, j & 31);
          if (j < 31) ya = fma(-Ls[j * kCsLd + lane], yj, ya);
          yb = fma(-Ls[j * kCsLd + lane + 32], yj, yb);
        }
        if (lane < bs) y[k0 + lane] = ya * rd[lane];
        if (lane + 32 < bs) y[k0 + 32 + lane] = yb * rd[lane + 32];
      }
      __syncthreads();
      if (k0 + kCsB < n) cs_stage_diag(L, ld, k0 + kCsB, min(kCsB, n - k0 - kCsB), true, Ls, rd);
    }
    grid.sync();
    if (k0 + kCsB >= n) break;                              // the same in every block
    if ((int)threadIdx.x < kCsB) blk[threadIdx.x] = __ldcg(y + k0 + threadIdx.x);
    __syncthreads();
    const int64_t nrest = n - (k0 + kCsB);                  // rows below the solved block
    if (b0) cs_update_rows(L, ld, k0, kCsB, true, 0, nrest < kCsB ? nrest : kCsB, kCsB, k0 + kCsB, 1, blk, red, y);
    else cs_update_rows(L, ld, k0, kCsB, true, kCsB + orow0, nrest, ostride, k0 + kCsB, 1, blk, red, y);
  }
  for (int64_t i = gtid; i < n; i += gthreads) x[i] = __ldcg(y + i);
  const int klast = n > 0 ? ((n - 1) / kCsB) * kCsB : 0;
  if (b0 && n > 0) cs_stage_diag(L, ld, klast, n - klast, false, Ls, rd);
  grid.sync();
  for (int k0 = klast; k0 >= 0 && n > 0; k0 -= kCsB) {      // L^T x = y
    const int bs = min(kCsB, n - k0);
    if (b0) {
      __syncthreads();
      if (warp == 0) {
        double xa = lane < bs ? __ldcg(x + k0 + lane) : 0.0;
        double xb = lane + 32 < bs ? __ldcg(x + k0 + 32 + lane) : 0.0;
        for (int j = bs - 1; j >= 0; --j) {                 // x_r -= (L[k0 + j, k0 + r] / L_jj) x_j
          const double xj = __shfl_sync(0xffffffffu, j < 32 ? xa : xb, j & 31);
          xa = fma(-Ls[lane * kCsLd + j], xj, xa);
          if (j > 32) xb = fma(-Ls[(lane + 32) * kCsLd + j], xj, xb);
        }
        if (lane < bs) x[k0 + lane] = xa * rd[lane];
        if (lane + 32 < bs) x[k0 + 32 + lane] = xb * rd[lane + 32];
      }
      __syncthreads();
      if (k0 > 0) cs_stage_diag(L, ld, k0 - kCsB, kCsB, false, Ls, rd);
    }
    grid.sync();
    if (k0 == 0) break;
    if ((int)threadIdx.x < kCsB) blk[threadIdx.x] = (int)threadIdx.x < bs ? __ldcg(x + k0 + threadIdx.x) : 0.0;
    __syncthreads();
    // row i = k0 - 1 - r: r < kCsB by block 0, the rest by the others
    if (b0) cs_update_rows(L, ld, k0, bs, false, 0, kCsB, kCsB, k0 - 1, -1, blk, red, x);
    else cs_update_rows(L, ld, k0, bs, false, kCsB + orow0, k0, ostride, k0 - 1, -1, blk, red, x);
  }
}
cudaError_t launch_chol_solve(const double* L, int n, int64_t ld, const double* b, double* x, double* y,
                              cudaStream_t s) {
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_chol_solve, kCsT, 0);
  const int blocks = std::max(2, std::max(1, std::min(per, 2)) * nsm);   // block 0 and at least one more
  void* args[] = {(void*)&L, &n, &ld, (void*)&b, &x, &y};
  note_launch();
  return cudaLaunchCooperativeKernel((const void*)k_chol_solve, blocks, kCsT, args, 0, s);
}

// ---------------------------------------------------------------------------- SIMT GEMM
// C(m, n) = sum_k A(m, k) B(k, n) with element strides; A(m,k) = A[m*sam + k*sak],
// B(k,n) = B[k*sbk + n*sbn].  64x64 tiles, 16-deep K slices, 4x4 per thread.
// FP32 products are summed in FP32 over 128-deep chunks and then in FP64.
// Output: out64 (double, partial per blockIdx.z at out64 + z*split_stride) or outT.
// Epilogue scales: rowscale[m] (double, nullable), colscale[n] (double, nullable).
template <typename T>
__global__ void __launch_bounds__(256) k_gemm(int64_t M, int64_t N, int64_t K, const T* __restrict__ A, int64_t sam,
                                              int64_t sak, const T* __restrict__ B, int64_t sbk, int64_t sbn,
                                              int64_t k_per_split, double* __restrict__ out64, int64_t split_stride,
                                              T* __restrict__ outT, int64_t scm, int64_t scn,
                                              const double* __restrict__ rowscale,
                                              const double* __restrict__ colscale, int accumulate) {
  constexpr int BM = 64, BN = 64, BK = 16;
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;
  const int64_t kb = (int64_t)blockIdx.z * k_per_split;
  const int64_t ke = min(K, kb + k_per_split);
  T acc[4][4];
  double acc64[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      acc[a][b] = T(0);
      acc64[a][b] = 0.0;
    }
  int slice = 0;
  for (int64_t k0 = kb; k0 < ke; k0 += BK) {
    // load A tile (BM x BK) and B tile (BK x BN): unit-stride dimension on consecutive threads
    for (int e = threadIdx.x; e < BM * BK; e += 256) {
      int mm, kk;
      if (sak == 1) { kk = e % BK; mm = e / BK; } else { mm = e % BM; kk = e / BM; }
      const int64_t gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < M && gk < ke) ? A[gm * sam + gk * sak] : T(0);
    }
    for (int e = threadIdx.x; e < BK * BN; e += 256) {
      int kk, nn;
      if (sbk == 1) { kk = e % BK; nn = e / BK; } else { nn = e % BN; kk = e / BN; }
      const int64_t gk = k0 + kk, gn = n0 + nn;
      Bs[kk][nn] = (gn < N && gk < ke) ? B[gk * sbk + gn * sbn] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = As[kk][ty + 16 * i];
        b[i] = Bs[kk][tx + 16 * i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
    if (sizeof(T) == 4 && (++slice & 7) == 0) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc64[i][j] += to_f64(acc[i][j]);
          acc[i][j] = T(0);
        }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
    const double rs = rowscale ? rowscale[gm] : 1.0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      double v = (acc64[i][j] + to_f64(acc[i][j])) * rs;
      if (colscale) v *= colscale[gn];
      if (out64) {
        double* o = out64 + (int64_t)blockIdx.z * split_stride + gm * scm + gn * scn;
        *o = accumulate ? *o + v : v;
      } else {
        T* o = outT + gm * scm + gn * scn;
        *o = accumulate ? (T)((double)*o + v) : (T)v;
      }
    }
  }
}

template <typename T>
void launch_gemm(const GemmArgs<T>& g, cudaStream_t s) {
  const int64_t kps = g.nsplit > 1 ? ((g.K + g.nsplit - 1) / g.nsplit + 15) / 16 * 16 : std::max<int64_t>(g.K, 1);
  const int nz = (int)((g.K + kps - 1) / kps);
  dim3 grid((unsigned)((g.M + 63) / 64), (unsigned)((g.N + 63) / 64), (unsigned)std::max(nz, 1));
  k_gemm<T><<<grid, 256, 0, s>>>(g.M, g.N, g.K, g.A, g.sam, g.sak, g.B, g.sbk, g.sbn, kps, g.out64, g.split_stride,
                                 g.outT, g.scm, g.scn, g.rowscale, g.colscale, g.accumulate); note_launch();
}
template void launch_gemm<float>(const GemmArgs<float>&, cudaStream_t);
template void launch_gemm<double>(const GemmArgs<double>&, cudaStream_t);

int gemm_splits(const GemmArgs<float>& g) {  // number of z-slices launch_gemm will use
  const int64_t kps = g.nsplit > 1 ? ((g.K + g.nsplit - 1) / g.nsplit + 15) / 16 * 16 : std::max<int64_t>(g.K, 1);
  return (int)std::max<int64_t>(1, (g.K + kps - 1) / kps);
}

// out[i] = sum_z part[z*stride + i] for i < n  (ordered, deterministic)
__global__ void k_sum_splits(const double* __restrict__ part, int nz, int64_t stride, int64_t n,
                             double* __restrict__ out) {
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += st) {
    double s = 0.0;
    for (int z = 0; z < nz; ++z) s += part[(int64_t)z * stride + i];
    out[i] = s;
  }
}
template <typename T>
__global__ void k_sum_splits_t(const double* __restrict__ part, int nz, int64_t stride, int64_t rows, int64_t cols,
                               int64_t ldp, T* __restrict__ out, int64_t ldo) {
  const int64_t n = rows * cols;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += st) {
    const int64_t c = e / rows, r = e - c * rows;
    double s = 0.0;
    for (int z = 0; z < nz; ++z) s += part[(int64_t)z * stride + r + c * ldp];
    out[r + c * ldo] = (T)s;
  }
}
void launch_sum_splits(const double* part, int nz, int64_t stride, int64_t n, double* out, cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
  k_sum_splits<<<blocks, 256, 0, s>>>(part, nz, stride, n, out); note_launch();
}
template <typename T>
void launch_sum_splits_t(const double* part, int nz, int64_t stride, int64_t rows, int64_t cols, int64_t ldp, T* out,
                         int64_t ldo, cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>((rows * cols + 255) / 256, 8192);
  k_sum_splits_t<T><<<blocks, 256, 0, s>>>(part, nz, stride, rows, cols, ldp, out, ldo); note_launch();
}
template void launch_sum_splits_t<float>(const double*, int, int64_t, int64_t, int64_t, int64_t, float*, int64_t,
                                         cudaStream_t);
template void launch_sum_splits_t<double>(const double*, int, int64_t, int64_t, int64_t, int64_t, double*, int64_t,
                                          cudaStream_t);

// ---------------------------------------------------------------------------- small elementwise helpers
// nu = scale * eps_m(||Y||_F), the spacing at ||Y||_F of a format with m explicit mantissa bits
// (2^(floor(log2 x) - m)), computed on the device from frob2 = ||Y||_F^2; stored in *nu_out.
__global__ void k_compute_nu(const double* frob2, int mant_bits, double scale, double* nu_out) {
  const double x = sqrt(*frob2);
  double nu = 0.0;
  if (x > 0.0 && isfinite(x)) {
    int e;
    frexp(x, &e);  // x = f 2^e, f in [0.5, 1): floor(log2 x) = e - 1
    nu = ldexp(1.0, e - 1 - mant_bits);
  }
  *nu_out = scale * nu;
}
void launch_compute_nu(const double* frob2, int mant_bits, double scale, double* nu_out, cudaStream_t s) {
  k_compute_nu<<<1, 1, 0, s>>>(frob2, mant_bits, scale, nu_out); note_launch();
}

template <typename T>
__global__ void k_frob2_part(const T* __restrict__ Y, int64_t ld, int64_t p, int ell, double* part) {
  __shared__ double red[32];
  double acc = 0.0;
  const int64_t n = p * ell;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
    const int64_t j = e / p, i = e - j * p;
    const double v = (double)Y[i + j * ld];
    acc += v * v;
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}
template <typename T>
void launch_frob2(const T* Y, int64_t ld, int64_t p, int ell, double* part, double* out, cudaStream_t s) {
  const int nb = (int)std::min<int64_t>((p * ell + 255) / 256, kRedBlocks);
  k_frob2_part<T><<<nb, 256, 0, s>>>(Y, ld, p, ell, part); note_launch();
  launch_sum_partials(part, nb, 1.0, out, s);
}
template void launch_frob2<float>(const float*, int64_t, int64_t, int, double*, double*, cudaStream_t);
template void launch_frob2<double>(const double*, int64_t, int64_t, int, double*, double*, cudaStream_t);

// dst = src + nu * Om  (p x ell, column-major, same ld; padding rows zero)
template <typename T>
__global__ void k_shift_add(const T* __restrict__ src, const T* __restrict__ Om, const double* __restrict__ nu,
                            T* __restrict__ dst, int64_t ld, int64_t p, int ell) {
  const double nv = *nu;
  const int64_t n = ld * ell;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
    const int64_t i = e % ld;
    dst[e] = i < p ? (T)((double)src[e] + nv * (double)Om[e]) : T(0);
  }
}
template <typename T>
void launch_shift_add(const T* src, const T* Om, const double* nu, T* dst, int64_t ld, int64_t p, int ell,
                      cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>((ld * ell + 255) / 256, 8192);
  k_shift_add<T><<<blocks, 256, 0, s>>>(src, Om, nu, dst, ld, p, ell); note_launch();
}
template void launch_shift_add<float>(const float*, const float*, const double*, float*, int64_t, int64_t, int,
                                      cudaStream_t);
template void launch_shift_add<double>(const double*, const double*, const double*, double*, int64_t, int64_t, int,
                                       cudaStream_t);

// dst (double) = Y (double) + nu Om (float), p x ell column-major, padding rows zero
__global__ void k_shift_add_mixed(const double* __restrict__ Y, const float* __restrict__ Om,
                                  const double* __restrict__ nu, double* __restrict__ dst, int64_t ld, int64_t p,
                                  int ell) {
  const double nv = *nu;
  const int64_t n = ld * ell;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
    const int64_t i = e % ld;
    dst[e] = i < p ? Y[e] + nv * (double)Om[e] : 0.0;
  }
}
void launch_shift_add_mixed(const double* Y, const float* Om, const double* nu, double* dst, int64_t ld, int64_t p,
                            int ell, cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>((ld * ell + 255) / 256, 8192);
  k_shift_add_mixed<<<blocks, 256, 0, s>>>(Y, Om, nu, dst, ld, p, ell); note_launch();
}

// M = (M + M^T) / 2 in place (n x n column-major)
__global__ void k_symmetrize(double* M, int n) {
  const int64_t total = (int64_t)n * n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
    const int i = (int)(e % n), j = (int)(e / n);
    if (i < j) {
      const double v = 0.5 * (M[i + (int64_t)j * n] + M[j + (int64_t)i * n]);
      M[i + (int64_t)j * n] = v;
      M[j + (int64_t)i * n] = v;
    }
  }
}
void launch_symmetrize(double* M, int n, cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>(((int64_t)n * n + 255) / 256, 4096);
  k_symmetrize<<<blocks, 256, 0, s>>>(M, n); note_launch();
}

// M[i][j] = M[j][i] for i < j: the upper triangle from the lower one (n x n column-major)
__global__ void k_mirror_lower(double* M, int n) {
  const int64_t total = (int64_t)n * n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
    const int i = (int)(e % n), j = (int)(e / n);
    if (i < j) M[e] = M[j + (int64_t)i * n];
  }
}
void launch_mirror_lower(double* M, int n, cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>(((int64_t)n * n + 255) / 256, 4096);
  k_mirror_lower<<<blocks, 256, 0, s>>>(M, n); note_launch();
}

// ---------------------------------------------------------------------------- triangular solve
// X (p x n, column-major, leading dimension ld) <- X L^{-T}, L lower (FP64, column-major n x n):
// blocked by 32-column panels, right-looking.  Per panel the rows are solved by forward
// substitution (x_j = (x_j - sum_{t<j} L[j,t] x_t) / L[j,j], one thread per row, FP64), then
// the trailing columns take the panel's contribution by a GEMM with W = -L^T
// (X[:, J'] += X[:, J] W[J, J']).  The GEMM runs in double-float arithmetic for double X (FP64
// accuracy on the FP32 pipes) and in FP32 for float X.
template <typename T>
__global__ void k_neg_transpose(const double* __restrict__ L, int n, T* __restrict__ W) {
  const int64_t total = (int64_t)n * n;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
    const int tt = (int)(e % n), j = (int)(e / n);  // W[tt + j n] = -L[j, tt] for j > tt
    W[e] = j > tt ? (T)(-L[j + (int64_t)tt * n]) : T(0);
  }
}

template <typename T>
__global__ void __launch_bounds__(128) k_trsm_panel(T* __restrict__ X, int64_t ld, int64_t p,
                                                   const double* __restrict__ L, int n, int b0, int bs) {
  __shared__ double Ls[32][33];
  __shared__ double rinv[32];
  for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
    const int i = e % 32, j = e / 32;
    Ls[i][j] = (i < bs && j <= i) ? L[(b0 + i) + (int64_t)(b0 + j) * n] : 0.0;
  }
  if (threadIdx.x < 32) rinv[threadIdx.x] = threadIdx.x < bs ? 1.0 / L[(int64_t)(b0 + threadIdx.x) * (n + 1)] : 0.0;
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // rows spread over the blocks first, so that few rows still occupy many SMs
  for (int64_t row = blockIdx.x + (int64_t)gridDim.x * threadIdx.x; row < p; row += stride) {
    T* xr = X + row + (int64_t)b0 * ld;
    double x[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) x[j] = j < bs ? (double)xr[(int64_t)j * ld] : 0.0;
#pragma unroll
    for (int j = 0; j < 32; ++j) {          // column-oriented substitution: x_j final, then eliminated
      x[j] *= rinv[j];
#pragma unroll
      for (int c = j + 1; c < 32; ++c) x[c] -= Ls[c][j] * x[j];
    }
#pragma unroll
    for (int j = 0; j < 32; ++j)
      if (j < bs) xr[(int64_t)j * ld] = (T)x[j];
  }
}

// Row-block form for double X: each CTA solves R whole rows in one launch (rows are independent),
// the rows held in shared memory as double-float pairs, column-major by column index.  Per
// 32-column block J: (1) x_J -= z_{<J} L_{J,<J}^T, double-float multiply-adds on packed f32x2
// lanes (two columns per instruction), L streamed in 32 x 32 chunks; (2) forward substitution in
// the 32 x 32 diagonal block in double-float (z_j = x_j / L_jj as a product with the FP64
// reciprocal's pair, then x_c -= L_cj z_j for c > j), one warp per row, lane = column.  The
// arithmetic carries ~2^-48 relative error per operation like the blocked form's GEMMs; the
// solve is one launch instead of two per 32-column panel.
constexpr int kTrsmThreads = 256;

// For FP32 X (the test matrix's CholeskyQR) the off-diagonal products run in plain FP32 on packed
// lanes with the high words of L, each 32-term chunk's sum added to a double-float accumulator
// (FP32 rounding over 32 terms, not over n), the diagonal blocks as for FP64 X.
template <int R, typename TX>
__global__ void __launch_bounds__(kTrsmThreads) k_trsm_rows(TX* __restrict__ X, int64_t ld, int64_t p,
                                                         const double* __restrict__ L, const float* __restrict__ LH,
                                                         const float* __restrict__ LL, int n) {
  constexpr bool F32 = sizeof(TX) == 4;
  static_assert(R == 16 || R == 32, "row block");
  constexpr int RP = R + 1;                            // padded column stride: no bank conflicts
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* Zh = reinterpret_cast<float*>(smem_raw);      // [n][RP]
  float* Zl = Zh + (size_t)n * RP;                     // [n][RP]
  // chunk of L as column pairs (j0 + c, j0 + c + 16), c < 16, of high and low words: [t - tc][c]
  __shared__ __align__(16) f2x LPh[32][16], LPl[32][16];
  __shared__ float Dh[32][33], Dl[32][33];             // diagonal block: [c][j]
  __shared__ float Rh[32], Rl[32];                     // 1 / L_jj as a pair
  const int tid = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * R;
  for (int64_t e = tid; e < (int64_t)n * R; e += kTrsmThreads) {
    const int r = (int)(e % R);
    const int64_t t = e / R;
    if constexpr (F32) {
      Zh[t * RP + r] = r0 + r < p ? X[r0 + r + t * ld] : 0.f;
      Zl[t * RP + r] = 0.f;
    } else {
      const double x = r0 + r < p ? X[r0 + r + t * ld] : 0.0;
      split_df(x, Zh[t * RP + r], Zl[t * RP + r]);
    }
  }
  const int tj = tid & 15, tr = tid >> 4;              // update: columns tj, tj + 16; rows tr (+16)
  const int warp = tid >> 5, lane = tid & 31;
  for (int j0 = 0; j0 < n; j0 += 32) {
    const int bw = min(32, n - j0);
    // diagonal block and reciprocals for step (2)
    for (int e = tid; e < 32 * 32; e += kTrsmThreads) {
      const int c = e & 31, j = e >> 5;
      const bool in = c < bw && j < c;
      const int64_t o = (j0 + c) + (int64_t)(j0 + j) * n;
      Dh[c][j] = in ? LH[o] : 0.f;
      Dl[c][j] = in && !F32 ? LL[o] : 0.f;            // FP32 X: L's high words only
    }
    if (tid < 32) {
      const double rv = tid < bw ? 1.0 / L[(int64_t)(j0 + tid) * (n + 1)] : 0.0;
      split_df(rv, Rh[tid], Rl[tid]);
    }
    // (1) x_J -= sum_{t < j0} z_t L_{J,t}; the next chunk of L is fetched into registers while
    // the current one is used
    DF2 acc[R / 16];
#pragma unroll
    for (int q = 0; q < R / 16; ++q) acc[q] = DF2{0ull, 0ull};
    float preh[4], prel[4];
    auto fetch = [&](int tc) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = tid + kTrsmThreads * u, jj = e & 31, tt = e >> 5;
        const int64_t o = (j0 + jj) + (int64_t)(tc + tt) * n;
        preh[u] = jj < bw ? LH[o] : 0.f;
        prel[u] = jj < bw ? LL[o] : 0.f;
      }
    };
    if (j0 > 0) fetch(0);
    for (int tc = 0; tc < j0; tc += 32) {
      __syncthreads();                                  // previous chunk consumed
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = tid + kTrsmThreads * u, jj = e & 31, tt = e >> 5;
        reinterpret_cast<float*>(&LPh[tt][jj & 15])[jj >> 4] = preh[u];
        reinterpret_cast<float*>(&LPl[tt][jj & 15])[jj >> 4] = prel[u];
      }
      __syncthreads();
      if (tc + 32 < j0) fetch(tc + 32);
      if constexpr (F32) {
        f2x cs[R / 16];
#pragma unroll
        for (int q = 0; q < R / 16; ++q) cs[q] = 0ull;
#pragma unroll 8
        for (int tt = 0; tt < 32; ++tt) {
          const f2x bh = LPh[tt][tj];
#pragma unroll
          for (int q = 0; q < R / 16; ++q) {
            const float zh = Zh[(size_t)(tc + tt) * RP + tr + 16 * q];
            cs[q] = fma2(pk2(zh, zh), bh, cs[q]);
          }
        }
#pragma unroll
        for (int q = 0; q < R / 16; ++q) {       // acc += chunk sum (TwoSum into the high word)
          const f2x t = add2(acc[q].hi, cs[q]);
          const f2x z = sub2(t, acc[q].hi);
          const f2x er = add2(sub2(acc[q].hi, sub2(t, z)), sub2(cs[q], z));
          acc[q].hi = t;
          acc[q].lo = add2(acc[q].lo, er);
        }
      } else {
#pragma unroll 4
      for (int tt = 0; tt < 32; ++tt) {
        const f2x bh = LPh[tt][tj];
        const f2x bl = LPl[tt][tj];
#pragma unroll
        for (int q = 0; q < R / 16; ++q) {
          const int r = tr + 16 * q;
          const float zh = Zh[(size_t)(tc + tt) * RP + r], zl = Zl[(size_t)(tc + tt) * RP + r];
          // acc += (zh + zl)(bh + bl): the product of the high words exactly, cross terms in lo
          const f2x ah = pk2(zh, zh), al = pk2(zl, zl);
          const f2x pn = mul2(ah ^ 0x8000000080000000ull, bh);
          f2x pe = fma2(ah, bh, pn);
          pe = fma2(ah, bl, pe);
          pe = fma2(al, bh, pe);
          const f2x t = sub2(acc[q].hi, pn);
          const f2x z = sub2(t, acc[q].hi);
          const f2x er = sub2(sub2(acc[q].hi, sub2(t, z)), add2(pn, z));
          acc[q].hi = t;
          acc[q].lo = add2(add2(acc[q].lo, pe), er);
        }
      }
      }
    }
    __syncthreads();                                    // diagonal block loaded, chunks done
    if (j0 > 0) {
#pragma unroll
      for (int q = 0; q < R / 16; ++q) {
        const int r = tr + 16 * q;
        DF a0, a1;
        df2_split(acc[q], a0, a1);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int c = tj + 16 * h;
          if (c < bw) {
            const size_t o = (size_t)(j0 + c) * RP + r;
            const DF a = h ? a1 : a0;
            const DF x = df_add(DF{Zh[o], Zl[o]}, DF{-a.hi, -a.lo});
            Zh[o] = x.hi;
            Zl[o] = x.lo;
          }
        }
      }
    }
    __syncthreads();
    // (2) substitution in the diagonal block: lane = column, the warp's rows interleaved
    {
      constexpr int NR = R / (kTrsmThreads / 32);
      DF x[NR];
#pragma unroll
      for (int q = 0; q < NR; ++q) {
        const size_t o = (size_t)(j0 + lane) * RP + warp + 8 * q;
        x[q] = lane < bw ? DF{Zh[o], Zl[o]} : DF{0.f, 0.f};
      }
      for (int j = 0; j < bw; ++j) {
        const float rh = Rh[j], rl = Rl[j], nlh = -Dh[lane][j], nll = -Dl[lane][j];
#pragma unroll
        for (int q = 0; q < NR; ++q) {
          const DF xj{__shfl_sync(0xffffffffu, x[q].hi, j), __shfl_sync(0xffffffffu, x[q].lo, j)};
          const DF zj = df_mul(xj, rh, rl);
          if (lane == j) {
            x[q] = zj;
          } else if (lane > j) {
            df_add_prod2(x[q], nlh, nll, zj.hi, zj.lo);   // x -= L_cj z_j
          }
        }
      }
      if (lane < bw) {
#pragma unroll
        for (int q = 0; q < NR; ++q) {
          const size_t o = (size_t)(j0 + lane) * RP + warp + 8 * q;
          Zh[o] = x[q].hi;
          Zl[o] = x[q].lo;
        }
      }
    }
    __syncthreads();
  }
  for (int64_t e = tid; e < (int64_t)n * R; e += kTrsmThreads) {
    const int r = (int)(e % R);
    const int64_t t = e / R;
    if (r0 + r < p) {
      if constexpr (F32) X[r0 + r + t * ld] = Zh[t * RP + r] + Zl[t * RP + r];
      else X[r0 + r + t * ld] = f32_to_f64(Zh[t * RP + r]) + f32_to_f64(Zl[t * RP + r]);
    }
  }
}

size_t trsm_rows_smem(int n, int R) { return (size_t)2 * n * (R + 1) * sizeof(float); }

// W: n x n scratch of T.
template <typename T>
void launch_trsm_lt(T* X, int64_t ld, int64_t p, int n, const double* L, T* W, cudaStream_t s) {
  {
    // one launch over row blocks while 16 rows of the solve fit in shared memory (two CTAs, 16
    // warps, per SM to hide the double-float chains' latency)
    constexpr int R = 16;
    const size_t smem = trsm_rows_smem(n, R);
    if (n >= 64 && smem <= 200 * 1024) {
      // L as double-float pairs once (W: n x n elements of T, at least n^2 floats; for FP32 X the
      // low words are not needed), so that no CTA converts FP64 in its inner loop
      float* LH = reinterpret_cast<float*>(W);
      float* LL = sizeof(T) == 8 ? LH + (int64_t)n * n : LH;
      if (sizeof(T) == 8) launch_split_df(L, LH, LL, (int64_t)n * n, (int64_t)n * n, s);
      else launch_f64_to_f32(L, LH, (int64_t)n * n, s);
      const unsigned grid = (unsigned)((p + R - 1) / R);
      static bool cfg = false;
      if (!cfg) {
        cudaFuncSetAttribute((const void*)k_trsm_rows<R, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cfg = true;
      }
      k_trsm_rows<R, T><<<grid, kTrsmThreads, smem, s>>>(X, ld, p, L, LH, LL, n);
      note_launch();
      return;
    }
  }
  const int blocks0 = (int)std::min<int64_t>(((int64_t)n * n + 255) / 256, 4096);
  k_neg_transpose<T><<<blocks0, 256, 0, s>>>(L, n, W); note_launch();
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  }
  const int pblocks = (int)std::min<int64_t>(std::max<int64_t>((p + 127) / 128, nsm), 4096);
  for (int b0 = 0; b0 < n; b0 += 32) {
    const int bs = std::min(32, n - b0);
    k_trsm_panel<T><<<pblocks, 128, 0, s>>>(X, ld, p, L, n, b0, bs); note_launch();
    const int c0 = b0 + bs;
    if (c0 >= n) break;
    if (std::is_same<T, double>::value) {
      GemmDfArgs<double, double> g;
      g.M = p; g.N = n - c0; g.K = bs;
      g.A = (const double*)X + (int64_t)b0 * ld; g.sam = 1; g.sak = ld;
      g.B = (const double*)W + b0 + (int64_t)c0 * n; g.sbk = 1; g.sbn = n;
      g.out64 = (double*)X + (int64_t)c0 * ld; g.scm = 1; g.scn = ld;
      g.accumulate = 1;
      launch_gemm_df<double, double>(g, s);
    } else {
      GemmArgs<T> g;
      g.M = p; g.N = n - c0; g.K = bs;
      g.A = X + (int64_t)b0 * ld; g.sam = 1; g.sak = ld;
      g.B = W + b0 + (int64_t)c0 * n; g.sbk = 1; g.sbn = n;
      g.outT = X + (int64_t)c0 * ld; g.scm = 1; g.scn = ld;
      g.accumulate = 1;
      launch_gemm<T>(g, s);
    }
  }
}
template void launch_trsm_lt<float>(float*, int64_t, int64_t, int, const double*, float*, cudaStream_t);
template void launch_trsm_lt<double>(double*, int64_t, int64_t, int, const double*, double*, cudaStream_t);

// ---------------------------------------------------------------------------- FP64 Cholesky
// Blocked right-looking Cholesky of the n x n SPD matrix A (column-major, lower triangle used
// and overwritten by L, A = L L^T) in one cooperative launch, two grid barriers per 16-wide
// panel (FP64 latency on GB300 is ~64 cycles per operation, ~1100 for a square root and a
// division, so the sequential chain through the diagonal blocks sets the time):
//   (a) all blocks solve the panel rows below the diagonal block (one thread per row, FP64);
//   (b) all blocks update the trailing lower triangle in 16 x 16 tiles staged in shared memory;
//       the block that updates the next diagonal tile factors it right away with one warp
//       (lane i holds row i, columns eliminated by shuffles).
// A non-positive or non-finite pivot sets kStatNotSpd; every block then leaves at the next barrier.
namespace {
constexpr int kCholNB = 16;        // short panels: the per-column FP64 chain is the critical path

// Factor the bs x bs diagonal block at (k0, k0) in place with warp 0 of the calling block.
__device__ void chol_diag_block(double* __restrict__ A, int n, int k0, int bs, int* __restrict__ status) {
  if (threadIdx.x >= 32) return;
  const int i = threadIdx.x;
  double a[kCholNB];
#pragma unroll
  for (int j = 0; j < kCholNB; ++j) a[j] = (i < bs && j <= i && j < bs) ? A[(k0 + i) + (int64_t)(k0 + j) * n] : 0.0;
  bool bad = false;
#pragma unroll
  for (int j = 0; j < kCholNB; ++j) {
    if (j < bs && !bad) {
      const double piv = __shfl_sync(0xffffffffu, a[j], j);
      if (!(piv > 0.0) || !isfinite(piv)) {
        bad = true;                         // uniform: every lane read the same pivot
      } else {
        const double r = rsqrt(piv), d = piv * r;   // one reciprocal square root per column
        a[j] = i == j ? d : (i > j ? a[j] * r : 0.0);
#pragma unroll
        for (int c = j + 1; c < kCholNB; ++c) {
          const double lcj = __shfl_sync(0xffffffffu, a[j], c);
          if (c < bs && i >= c) a[c] -= a[j] * lcj;
        }
      }
    }
  }
  if (bad) {
    if (i == 0) atomicOr(status, kStatNotSpd);
    return;
  }
#pragma unroll
  for (int j = 0; j < kCholNB; ++j)
    if (i < bs && j <= i && j < bs) A[(k0 + i) + (int64_t)(k0 + j) * n] = a[j];
}
}  // namespace

__global__ void __launch_bounds__(256) k_cholesky(double* __restrict__ A, int n, int* __restrict__ status) {
  constexpr int NB = kCholNB;
  cg::grid_group grid = cg::this_grid();
  __shared__ double D[NB][NB + 1];
  __shared__ double rinv[NB];
  __shared__ double Pi[NB][NB + 1], Pj[NB][NB + 1];
  const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
  if (blockIdx.x == 0) chol_diag_block(A, n, 0, min(NB, n), status);
  grid.sync();
  for (int k0 = 0; k0 < n; k0 += NB) {
    if (*((volatile int*)status) & kStatNotSpd) return;
    const int bs = min(NB, n - k0);
    const int r0 = k0 + bs, m = n - r0;
    if (m <= 0) break;
    // (a) panel rows: L[i, k0:k0+bs] = A[i, k0:k0+bs] L_kk^{-T}
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
      const int i = e % NB, j = e / NB;
      D[i][j] = (i < bs && j <= i) ? A[(k0 + i) + (int64_t)(k0 + j) * n] : 0.0;
    }
    if (threadIdx.x < NB) rinv[threadIdx.x] = threadIdx.x < bs ? 1.0 / A[(int64_t)(k0 + threadIdx.x) * (n + 1)] : 0.0;
    __syncthreads();
    // rows spread over the blocks first (few rows: one or two per SM)
    for (int64_t i = r0 + blockIdx.x + (int64_t)gridDim.x * threadIdx.x; i < n; i += gthreads) {
      double x[NB];
#pragma unroll
      for (int j = 0; j < NB; ++j) x[j] = j < bs ? A[i + (int64_t)(k0 + j) * n] : 0.0;
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        x[j] *= rinv[j];
#pragma unroll
        for (int c = j + 1; c < NB; ++c) x[c] -= D[c][j] * x[j];
      }
#pragma unroll
      for (int j = 0; j < NB; ++j)
        if (j < bs) A[i + (int64_t)(k0 + j) * n] = x[j];
    }
    grid.sync();
    // (b) trailing update of the lower triangle in 32 x 32 tiles: A[I, J] -= P_I P_J^T with
    //     P = L[:, k0:k0+bs]; tile (0, 0) (the next diagonal block) goes to block 0 first
    const int nt = (m + NB - 1) / NB;
    const int ntiles = nt * (nt + 1) / 2;
    for (int tIdx = blockIdx.x; tIdx < ntiles; tIdx += gridDim.x) {
      int ti = 0;                           // tile (ti, tj), tj <= ti, in row-major lower order
      while ((ti + 1) * (ti + 2) / 2 <= tIdx) ++ti;
      const int tj = tIdx - ti * (ti + 1) / 2;
      const int ri = r0 + ti * NB, rj = r0 + tj * NB;
      __syncthreads();
      for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
        const int r = e % NB, c = e / NB;
        Pi[r][c] = (ri + r < n && c < bs) ? A[(ri + r) + (int64_t)(k0 + c) * n] : 0.0;
        Pj[r][c] = (rj + r < n && c < bs) ? A[(rj + r) + (int64_t)(k0 + c) * n] : 0.0;
      }
      __syncthreads();
      const int r = threadIdx.x % NB;
#pragma unroll
      for (int q = 0; q < NB * NB / 256; ++q) {
        const int c = threadIdx.x / NB + q * (256 / NB);
        const int gi = ri + r, gj = rj + c;
        if (gi < n && gj < n && gj <= gi) {
          double s = 0.0;
#pragma unroll
          for (int t = 0; t < NB; ++t) s += Pi[r][t] * Pj[c][t];
          A[gi + (int64_t)gj * n] -= s;
        }
      }
      if (tIdx == 0) {                      // the next diagonal block is final: factor it
        __syncthreads();
        chol_diag_block(A, n, r0, min(NB, m), status);
      }
    }
    grid.sync();
  }
}

static int coop_blocks(const void* kernel, int threads, size_t smem) {
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem);
  return std::max(1, std::min(per, 2)) * nsm;
}

cudaError_t launch_cholesky(double* A, int n, int* status, cudaStream_t s) {
  const int blocks = coop_blocks((const void*)k_cholesky, 256, 0);
  void* args[] = {&A, &n, &status};
  note_launch();
  return cudaLaunchCooperativeKernel((const void*)k_cholesky, blocks, 256, args, 0, s);
}

// W = V diag(1/sigma) (column scale), lam = max(0, sigma^2 - nu) and 1/sigma for the U GEMM.
__global__ void k_nystrom_lambda(const double* __restrict__ sig2, const double* __restrict__ nu, int n,
                                 double* __restrict__ lam, double* __restrict__ inv_sigma) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const double s2 = sig2[j];
    lam[j] = fmax(0.0, s2 - *nu);
    inv_sigma[j] = s2 > 0.0 ? 1.0 / sqrt(s2) : 0.0;
  }
}
void launch_nystrom_lambda(const double* sig2, const double* nu, int n, double* lam, double* inv_sigma,
                           cudaStream_t s) {
  k_nystrom_lambda<<<(n + 255) / 256, 256, 0, s>>>(sig2, nu, n, lam, inv_sigma); note_launch();
}

// mu = gamma * eps64 * lam[0] (Alg. 4), or the fixed value when fixed_mu > 0
// mu: the fixed value if positive, else gamma eps64 lambda_hat_1 (Alg. 4), raised to c L^2 when the
// adaptive damping of Sec. 5 is on (c > 0; loss = L(theta) on the device)
__global__ void k_set_mu(const double* __restrict__ lam, double fixed_mu, double gamma, const double* __restrict__ loss,
                         double c, double* __restrict__ mu) {
  double m = fixed_mu > 0.0 ? fixed_mu : gamma * 0x1p-52 * lam[0];
  if (!(fixed_mu > 0.0) && c > 0.0) m = fmax(m, c * (*loss) * (*loss));
  *mu = m;
}
void launch_set_mu(const double* lam, double fixed_mu, double gamma, const double* loss, double c, double* mu,
                   cudaStream_t s) {
  k_set_mu<<<1, 1, 0, s>>>(lam, fixed_mu, gamma, loss, c, mu); note_launch();
}

}  // namespace ngd
