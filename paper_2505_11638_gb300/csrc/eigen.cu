// FP64 symmetric eigen-decomposition of the l x l Nystrom core S = B^T B (App. A: the thin SVD
// of B, read as eig(B^T B) and U = B V Sigma^{-1}).
//
// GB300 has few FP64 units per SM (~8 flop/clk) and a grid-wide barrier costs ~1.2 us, so the
// solver keeps the number of dependent steps and the FP64 work per SM low:
//   1. Householder tridiagonalization S = Q T Q^T in one cooperative kernel: per column two
//      grid barriers; the symmetric matrix-vector product and the rank-2 update are spread
//      over 32 x 32 tiles of the trailing block on all SMs (deterministic partial sums).
//   2. Eigenvalues of T by multisection (a half-warp per eigenvalue, 16 Sturm counts per step,
//      three FP64 operations per step of the recurrence, two eigenvalues per block so that the
//      FP64 pipes of all SMs take part).
//   3. Eigenvectors of T by one twisted factorization per eigenvalue (one thread each, its
//      recurrences' operands in shared memory):
//      T - lambda I = L+ D+ L+^T = U- D- U-^T, twist index r = argmin |gamma_r|,
//      gamma_r = D+_r + D-_r - (d_r - lambda), z_r = 1 and the two bidiagonal recurrences.
//   4. V = Q Z by applying the reflectors to the columns of Z (one warp per column in FP64; in
//      FP32 contexts one warp per two columns in double-float on packed f32x2 lanes).
//   5. V is re-orthonormalised.  Twisted vectors of well-separated eigenvalues are already
//      orthogonal to eps ||T|| / gap (measured on the 5-D Poisson trajectory at ell = 500:
//      max |V^T V - I| ~ 1e-12), and then Newton-Schulz steps V <- V (3 I - V^T V) / 2 (one or
//      two) take V to its orthonormal polar factor, moving each vector by about half its overlaps
//      with the others: two small GEMMs per step instead of a Cholesky factorization and a
//      triangular solve, both chains of l dependent steps.  Eigenvalues closer than the rounding
//      of S (the noise floor of the Nystrom core) can give (nearly) equal vectors; when
//      ||V^T V - I||_F exceeds 1/2 the solver takes shifted CholeskyQR followed by two plain passes
//      instead (Fukaya, Kannan, Nakatsukasa, Yamamoto, Yanagisawa, SIAM J. Sci. Comput. 2020),
//      which turns them into an orthonormal basis of their joint invariant subspace.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>

#include "df.cuh"
#include "linalg.cuh"

namespace cg = cooperative_groups;

namespace ngd {

namespace {

__device__ __forceinline__ double wsum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------- 1. tridiagonalization
// A (n x n, column-major, symmetric, destroyed).  Outputs: d (n), e (n-1), tau (n), the
// Householder vectors Vh[k*n + i] (i = 0..n-k-2, the part acting on rows k+1..n-1).
// Scratch: ppart (ntm x 32 ntm), tdot (ntm x ntm), ntm = ceil((n-1)/32).
__global__ void __launch_bounds__(256) k_tridiag(double* __restrict__ A, int n, double* __restrict__ d,
                                                 double* __restrict__ e, double* __restrict__ tau,
                                                 double* __restrict__ Vh, double* __restrict__ ppart,
                                                 double* __restrict__ tdot) {
  const int64_t pst = (int64_t)32 * ((n - 1 + 31) / 32);   // row stride of the tile partials
  cg::grid_group grid = cg::this_grid();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* v = reinterpret_cast<double*>(smem_raw);  // [n]
  __shared__ double red[8];
  __shared__ double s_alpha, s_tau, s_K;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gwarp = blockIdx.x * (blockDim.x >> 5) + warp;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;                 // trailing block rows/cols k+1 .. n-1
    const double* col = A + (int64_t)k * n + (k + 1);
    // (a) Householder vector of column k (every block, identical arithmetic)
    double s2 = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      const double x = col[i];
      v[i] = x;
      s2 += x * x;
    }
    s2 = wsum_d(s2);
    if (lane == 0) red[warp] = s2;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      const double x0 = v[0];
      const double sig = sqrt(t);
      double alpha, tu, v0;
      if (t - x0 * x0 <= 0.0) {          // nothing below the subdiagonal: H = I
        alpha = x0;
        tu = 0.0;
        v0 = 0.0;
      } else {
        alpha = x0 >= 0.0 ? -sig : sig;
        v0 = x0 - alpha;
        tu = 2.0 / (2.0 * (t + fabs(x0) * sig));
      }
      v[0] = v0;
      s_alpha = alpha;
      s_tau = tu;
    }
    __syncthreads();
    const double tk = s_tau;
    if (blockIdx.x == 0) {
      if (threadIdx.x == 0) {
        d[k] = A[(int64_t)k * n + k];
        e[k] = s_alpha;
        tau[k] = tk;
      }
      for (int i = threadIdx.x; i < m; i += blockDim.x) Vh[(int64_t)k * n + i] = v[i];
    }
    if (tk == 0.0) {          // uniform across the grid: every block computed the same tau
      grid.sync();
      continue;
    }
    const int nt = (m + 31) / 32;
    const double* B = A + (int64_t)(k + 1) * n + (k + 1);   // trailing block, leading dimension n
    // (b) partial products of A22 v per 32 x 32 tile, and v^T A22 v per tile
    for (int t = gwarp; t < nt * nt; t += nwarps) {
      const int ti = t % nt, tj = t / nt;
      const int i = ti * 32 + lane;
      double acc = 0.0;
      if (i < m) {
        const int j1 = min(m, tj * 32 + 32);
        for (int j = tj * 32; j < j1; ++j) acc += B[i + (int64_t)j * n] * v[j];
      }
      ppart[(int64_t)tj * pst + i] = acc;   // rows >= m hold 0
      const double dt = wsum_d(i < m ? v[i] * acc : 0.0);
      if (lane == 0) tdot[t] = dt;
    }
    grid.sync();
    // (c) p = tau A22 v, K = tau/2 v^T p, w = p - K v;  A22 -= v w^T + w v^T
    if (threadIdx.x == 0) {
      double vav = 0.0;
      for (int t = 0; t < nt * nt; ++t) vav += tdot[t];
      s_K = 0.5 * tk * tk * vav;
    }
    __syncthreads();
    const double K = s_K;
    for (int t = gwarp; t < nt * nt; t += nwarps) {
      const int ti = t % nt, tj = t / nt;
      const int i = ti * 32 + lane, jl = tj * 32 + lane;
      double pi = 0.0, pj = 0.0;
      for (int c = 0; c < nt; ++c) {
        pi += ppart[(int64_t)c * pst + i];
        pj += ppart[(int64_t)c * pst + jl];
      }
      const double vi = i < m ? v[i] : 0.0, vj = jl < m ? v[jl] : 0.0;
      const double wi = tk * pi - K * vi, wj = tk * pj - K * vj;
      const int jn = min(32, m - tj * 32);   // uniform across the warp
      for (int jj = 0; jj < jn; ++jj) {
        const double wjj = __shfl_sync(0xffffffffu, wj, jj);
        const double vjj = __shfl_sync(0xffffffffu, vj, jj);
        if (i < m) {
          double* a = A + (int64_t)(k + 1 + tj * 32 + jj) * n + (k + 1 + i);
          *a -= vi * wjj + wi * vjj;
        }
      }
    }
    grid.sync();
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (n >= 2) {
      d[n - 2] = A[(int64_t)(n - 2) * n + (n - 2)];
      d[n - 1] = A[(int64_t)(n - 1) * n + (n - 1)];
      e[n - 2] = A[(int64_t)(n - 2) * n + (n - 1)];
    } else {
      d[0] = A[0];
    }
  }
}

// Distributed variant for n small enough that each block can hold its share of A: column j
// lives in the shared memory of block j % G for the whole reduction, so per column only the
// Householder vector v and p = tau A22 v cross the grid (through L2), with one grid barrier and
// one flag per column:
//   every block: wait for flag k (reflector k published), p_j = tau A[:, j] . v for its columns
//                j > k (A symmetric), partial v . p                               -> barrier
//   every block: K = tau/2 v . p, w = p - K v; the owner of column k + 1 updates that column
//                first, forms reflector k + 1 and sets flag k + 1 (look-ahead), then every block
//                updates the rest of its columns, A[:, j] -= v w_j + w v_j.
// The vectors, partial products and block partials are double-buffered by the parity of k, so a
// block that runs ahead into step k + 1 never overwrites what a slower block still reads for
// step k.  A flag wait gives up after kEigWaitCycles clock cycles (TIMEOUT in *status, after
// which no block waits again; the kernel still passes every barrier, so it cannot hang).
// vbuf, pbuf: 2 n doubles each; red: 2 G doubles; flags: n words, zero at launch.
namespace {

constexpr long long kEigWaitCycles = 4000000000LL;

// Householder reflector of the trailing part of column k held in col (full column, length n);
// v goes to vout (and Vh), tau / d / e to their arrays.
__device__ void house_from_col(const double* __restrict__ col, int n, int k, double* __restrict__ d,
                               double* __restrict__ e, double* __restrict__ tau, double* __restrict__ Vh,
                               double* __restrict__ vout, double* red8, double* s_bc) {
  const int m = n - k - 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double s2 = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double x = col[k + 1 + i];
    s2 = fma(x, x, s2);
  }
  s2 = wsum_d(s2);
  if (lane == 0) red8[warp] = s2;
  __syncthreads();
  if (warp == 0) {
    double tsum = lane < (int)(blockDim.x >> 5) ? red8[lane] : 0.0;
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) tsum += __shfl_xor_sync(0xffffffffu, tsum, o);
    if (lane == 0) {
      const double x0 = col[k + 1];
      const double sig = sqrt(tsum);
      double alpha, tu, v0;
      if (tsum - x0 * x0 <= 0.0) {      // nothing below the subdiagonal: H = I
        alpha = x0;
        tu = 0.0;
        v0 = 0.0;
      } else {
        alpha = x0 >= 0.0 ? -sig : sig;
        v0 = x0 - alpha;
        tu = 1.0 / (tsum + fabs(x0) * sig);
      }
      d[k] = col[k];
      e[k] = alpha;
      __stcg(tau + k, tu);
      s_bc[0] = v0;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double vi = i == 0 ? s_bc[0] : col[k + 1 + i];
    __stcg(vout + i, vi);
    Vh[(int64_t)k * n + i] = vi;
  }
}

__device__ __forceinline__ void publish_flag(unsigned* flag) {
  __syncthreads();                                  // every v / tau store of the block issued
  if (threadIdx.x == 0) {
    __threadfence();
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(flag), "r"(1u) : "memory");
  }
}

__device__ __forceinline__ void wait_flag(const unsigned* flag, int* status) {
  if (threadIdx.x == 0 && !(*(volatile int*)status & kStatTimeout)) {   // after a timeout: no more waits
    const long long t0 = clock64();
    unsigned v = 0;
    while (true) {
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
      if (v) break;
      if (clock64() - t0 > kEigWaitCycles) {
        atomicOr(status, kStatTimeout);
        break;
      }
    }
  }
  __syncthreads();
}

}  // namespace

__global__ void __launch_bounds__(256) k_tridiag_dist(const double* __restrict__ A, int n, double* __restrict__ d,
                                                      double* __restrict__ e, double* __restrict__ tau,
                                                      double* __restrict__ Vh, double* __restrict__ vbuf,
                                                      double* __restrict__ pbuf, double* __restrict__ red,
                                                      unsigned* __restrict__ flags, int* __restrict__ status) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int G = gridDim.x, b = blockIdx.x;
  const int ncl = (n + G - 1) / G;
  double* cols = reinterpret_cast<double*>(smem_raw);    // [ncl][n]
  double* vs = cols + (int64_t)ncl * n;                   // [n]
  double* ws = vs + n;                                    // [n]
  __shared__ double red8[8];
  __shared__ double s_bc[2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int s = 0; s < ncl; ++s) {
    const int j = b + s * G;
    for (int i = threadIdx.x; i < n; i += blockDim.x) cols[(int64_t)s * n + i] = j < n ? A[i + (int64_t)j * n] : 0.0;
  }
  __syncthreads();
  if (n >= 3 && b == 0) {
    house_from_col(cols, n, 0, d, e, tau, Vh, vbuf, red8, s_bc);
    publish_flag(flags);
  }
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;
    const int par = k & 1;
    const double* vk = vbuf + (int64_t)par * n;
    double* pk = pbuf + (int64_t)par * n;
    double* rk = red + (int64_t)par * G;
    if (k % G != b) wait_flag(flags + k, status);
    for (int i = threadIdx.x; i < m; i += blockDim.x) vs[i] = __ldcg(vk + i);   // with tau: one round trip
    const double tk = __ldcg(tau + k);
    const int s_first = (k + 1 - b + G - 1) / G;          // first local slot with column j > k
    __syncthreads();
    if (tk != 0.0) {                                      // uniform: every block reads the same tau
      // p_j = tau A[k+1:, j] . v for owned columns j > k, one warp per column
      double part = 0.0;
      for (int s = s_first + warp; s < ncl; s += (int)(blockDim.x >> 5)) {
        const int j = b + s * G;
        if (j >= n) break;
        const double* col = cols + (int64_t)s * n + k + 1;
        double a0 = 0.0, a1 = 0.0;
        int i = lane;
        for (; i + 32 < m; i += 64) {
          a0 = fma(col[i], vs[i], a0);
          a1 = fma(col[i + 32], vs[i + 32], a1);
        }
        if (i < m) a0 = fma(col[i], vs[i], a0);
        const double pj = tk * wsum_d(a0 + a1);
        if (lane == 0) {
          __stcg(pk + (j - k - 1), pj);
          part = fma(vs[j - k - 1], pj, part);
        }
      }
      if (lane == 0) red8[warp] = part;
      __syncthreads();
      if (warp == 0) {
        double sb = lane < (int)(blockDim.x >> 5) ? red8[lane] : 0.0;
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) sb += __shfl_xor_sync(0xffffffffu, sb, o);
        if (lane == 0) __stcg(rk + b, sb);
      }
    }
    grid.sync();
    const bool next = k + 3 < n;
    const int own_next = next && (k + 1) % G == b;
    if (tk != 0.0) {
      // K = tau/2 v . p (summed over blocks in block order), w = p - K v
      if (warp == 0) {
        double sv = 0.0;
        for (int q = lane; q < G; q += 32) sv += __ldcg(rk + q);
        sv = wsum_d(sv);
        if (lane == 0) s_bc[1] = 0.5 * tk * sv;
      }
      for (int i = threadIdx.x; i < m; i += blockDim.x) ws[i] = __ldcg(pk + i);
      __syncthreads();
      const double K = s_bc[1];
      for (int i = threadIdx.x; i < m; i += blockDim.x) ws[i] = fma(-K, vs[i], ws[i]);
      __syncthreads();
      if (own_next) {                                     // look-ahead: column k + 1 first
        double* col = cols + (int64_t)((k + 1) / G) * n + k + 1;
        const double wj = ws[0], vj = vs[0];
        for (int i = threadIdx.x; i < m; i += blockDim.x) col[i] -= vs[i] * wj + ws[i] * vj;
        __syncthreads();
      }
    }
    if (own_next) {
      house_from_col(cols + (int64_t)((k + 1) / G) * n, n, k + 1, d, e, tau, Vh, vbuf + (int64_t)(par ^ 1) * n,
                     red8, s_bc);
      publish_flag(flags + k + 1);
    }
    if (tk != 0.0) {
      for (int s = s_first; s < ncl; ++s) {
        const int j = b + s * G;
        if (j >= n) break;
        if (own_next && j == k + 1) continue;
        double* col = cols + (int64_t)s * n + k + 1;
        const double wj = ws[j - k - 1], vj = vs[j - k - 1];
        for (int i = threadIdx.x; i < m; i += blockDim.x) col[i] -= vs[i] * wj + ws[i] * vj;
      }
    }
    __syncthreads();
  }
  // the last 2 x 2 block
  if (threadIdx.x == 0) {
    if (n >= 2) {
      if ((n - 2) % G == b) {
        const double* c = cols + (int64_t)((n - 2) / G) * n;
        d[n - 2] = c[n - 2];
        e[n - 2] = c[n - 1];
      }
      if ((n - 1) % G == b) d[n - 1] = cols[(int64_t)((n - 1) / G) * n + n - 1];
    } else if (b == 0) {
      d[0] = cols[0];
    }
  }
}


// Double-float form of k_tridiag_dist for FP32 contexts (the Nystrom core FP64-accurate to
// ~2^-48): the columns, v, p and w as FP32 pairs, the matrix-vector products and rank-2 updates on
// the FP32 pipes.  With one block per SM each block owns ~n / 152 columns, and in FP64 their
// products and updates cost ~1.5 us per column of GB300's narrow FP64 pipe.  The reflector's
// scalars (norm, sigma, tau) and the cross-block sum K stay FP64; the outputs (d, e, tau, Vh) are
// FP64.  Same protocol, buffers and bounded waits as k_tridiag_dist (vbuf and pbuf hold pairs).
namespace {

__device__ __forceinline__ DF ld_df(const DF* p) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return DF{v.x, v.y};
}
__device__ __forceinline__ void st_df(DF* p, DF v) { __stcg(reinterpret_cast<float2*>(p), make_float2(v.hi, v.lo)); }

__device__ __forceinline__ DF dsplit(double x) {
  DF r;
  split_df(x, r.hi, r.lo);
  return r;
}

// hi + lo renormalised (|lo| <= half an FP32 unit of hi): a stored pair that later enters a
// product whose lo x lo term is dropped must not carry a low word grown by cancellations
__device__ __forceinline__ DF df_norm(DF a) {
  float s, e;
  two_sum(a.hi, a.lo, s, e);
  return DF{s, e};
}

__device__ void house_from_col_df(const DF* __restrict__ col, int n, int k, double* __restrict__ d,
                                  double* __restrict__ e, double* __restrict__ tau, double* __restrict__ Vh,
                                  DF* __restrict__ vout, DF* red8, double* s_bc) {
  const int m = n - k - 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  DF s2{0.f, 0.f};
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const DF x = col[k + 1 + i];
    df_add_prod2(s2, x.hi, x.lo, x.hi, x.lo);
  }
  s2 = warp_sum_df(s2);
  if (lane == 0) red8[warp] = s2;
  __syncthreads();
  if (warp == 0) {
    DF t = lane < (int)(blockDim.x >> 5) ? red8[lane] : DF{0.f, 0.f};
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) t = df_add(t, shfl_xor_df(t, o));
    if (lane == 0) {
      const double tsum = df_to_double(t);
      const double x0 = df_to_double(col[k + 1]);
      const double sig = sqrt(tsum);
      double alpha, tu, v0;
      if (tsum - x0 * x0 <= 0.0) {      // nothing below the subdiagonal: H = I
        alpha = x0;
        tu = 0.0;
        v0 = 0.0;
      } else {
        alpha = x0 >= 0.0 ? -sig : sig;
        v0 = x0 - alpha;
        tu = 1.0 / (tsum + fabs(x0) * sig);
      }
      d[k] = df_to_double(col[k]);
      e[k] = alpha;
      __stcg(tau + k, tu);
      s_bc[0] = v0;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const DF vi = i == 0 ? dsplit(s_bc[0]) : col[k + 1 + i];
    st_df(vout + i, vi);
    Vh[(int64_t)k * n + i] = i == 0 ? s_bc[0] : df_to_double(vi);
  }
}

}  // namespace

__global__ void __launch_bounds__(256) k_tridiag_dist_df(const double* __restrict__ A, int n, double* __restrict__ d,
                                                         double* __restrict__ e, double* __restrict__ tau,
                                                         double* __restrict__ Vh, double* __restrict__ vbuf_,
                                                         double* __restrict__ pbuf_, double* __restrict__ red,
                                                         unsigned* __restrict__ flags, int* __restrict__ status) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int G = gridDim.x, b = blockIdx.x;
  const int ncl = (n + G - 1) / G;
  DF* cols = reinterpret_cast<DF*>(smem_raw);            // [ncl][n]
  DF* vs = cols + (int64_t)ncl * n;                       // [n]
  DF* ws = vs + n;                                        // [n]
  DF* vbuf = reinterpret_cast<DF*>(vbuf_);                // [2][n]
  DF* pbuf = reinterpret_cast<DF*>(pbuf_);                // [2][n]
  __shared__ DF red8[8];
  __shared__ double s_bc[2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int s = 0; s < ncl; ++s) {
    const int j = b + s * G;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
      cols[(int64_t)s * n + i] = j < n ? dsplit(A[i + (int64_t)j * n]) : DF{0.f, 0.f};
  }
  __syncthreads();
  if (n >= 3 && b == 0) {
    house_from_col_df(cols, n, 0, d, e, tau, Vh, vbuf, red8, s_bc);
    publish_flag(flags);
  }
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;
    const int par = k & 1;
    const DF* vk = vbuf + (int64_t)par * n;
    DF* pk = pbuf + (int64_t)par * n;
    double* rk = red + (int64_t)par * G;
    if (k % G != b) wait_flag(flags + k, status);
    for (int i = threadIdx.x; i < m; i += blockDim.x) vs[i] = ld_df(vk + i);   // with tau: one round trip
    const double tk = __ldcg(tau + k);
    const int s_first = (k + 1 - b + G - 1) / G;          // first local slot with column j > k
    __syncthreads();
    if (tk != 0.0) {                                      // uniform: every block reads the same tau
      const DF tkd = dsplit(tk);
      // p_j = tau A[k+1:, j] . v for owned columns j > k, one warp per column
      DF part{0.f, 0.f};
      for (int s = s_first + warp; s < ncl; s += (int)(blockDim.x >> 5)) {
        const int j = b + s * G;
        if (j >= n) break;
        const DF* col = cols + (int64_t)s * n + k + 1;
        DF a0{0.f, 0.f}, a1{0.f, 0.f};
        int i = lane;
        for (; i + 32 < m; i += 64) {
          df_add_prod2(a0, col[i].hi, col[i].lo, vs[i].hi, vs[i].lo);
          df_add_prod2(a1, col[i + 32].hi, col[i + 32].lo, vs[i + 32].hi, vs[i + 32].lo);
        }
        if (i < m) df_add_prod2(a0, col[i].hi, col[i].lo, vs[i].hi, vs[i].lo);
        const DF dot = warp_sum_df(df_add(a0, a1));
        const DF pj = df_mul(dot, tkd.hi, tkd.lo);
        if (lane == 0) {
          st_df(pk + (j - k - 1), pj);
          const DF vj = vs[j - k - 1];
          df_add_prod2(part, vj.hi, vj.lo, pj.hi, pj.lo);
        }
      }
      if (lane == 0) red8[warp] = part;
      __syncthreads();
      if (warp == 0) {
        DF sb = lane < (int)(blockDim.x >> 5) ? red8[lane] : DF{0.f, 0.f};
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) sb = df_add(sb, shfl_xor_df(sb, o));
        if (lane == 0) __stcg(rk + b, df_to_double(sb));
      }
    }
    grid.sync();
    const bool next = k + 3 < n;
    const int own_next = next && (k + 1) % G == b;
    if (tk != 0.0) {
      // K = tau/2 v . p (summed over blocks in block order, FP64), w = p - K v
      if (warp == 0) {
        double sv = 0.0;
        for (int q = lane; q < G; q += 32) sv += __ldcg(rk + q);
        sv = wsum_d(sv);
        if (lane == 0) s_bc[1] = 0.5 * tk * sv;
      }
      for (int i = threadIdx.x; i < m; i += blockDim.x) ws[i] = ld_df(pk + i);
      __syncthreads();
      const DF nK = dsplit(-s_bc[1]);
      for (int i = threadIdx.x; i < m; i += blockDim.x) {
        DF w = ws[i];
        df_add_prod2(w, nK.hi, nK.lo, vs[i].hi, vs[i].lo);
        ws[i] = df_norm(w);
      }
      __syncthreads();
      if (own_next) {                                     // look-ahead: column k + 1 first
        DF* col = cols + (int64_t)((k + 1) / G) * n + k + 1;
        const DF wj = ws[0], vj = vs[0];
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
          DF c = col[i];
          df_add_prod2(c, -vs[i].hi, -vs[i].lo, wj.hi, wj.lo);
          df_add_prod2(c, -ws[i].hi, -ws[i].lo, vj.hi, vj.lo);
          col[i] = df_norm(c);
        }
        __syncthreads();
      }
    }
    if (own_next) {
      house_from_col_df(cols + (int64_t)((k + 1) / G) * n, n, k + 1, d, e, tau, Vh, vbuf + (int64_t)(par ^ 1) * n,
                        red8, s_bc);
      publish_flag(flags + k + 1);
    }
    if (tk != 0.0) {
      for (int s = s_first; s < ncl; ++s) {
        const int j = b + s * G;
        if (j >= n) break;
        if (own_next && j == k + 1) continue;
        DF* col = cols + (int64_t)s * n + k + 1;
        const DF wj = ws[j - k - 1], vj = vs[j - k - 1];
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
          DF c = col[i];
          df_add_prod2(c, -vs[i].hi, -vs[i].lo, wj.hi, wj.lo);
          df_add_prod2(c, -ws[i].hi, -ws[i].lo, vj.hi, vj.lo);
          col[i] = df_norm(c);
        }
      }
    }
    __syncthreads();
  }
  // the last 2 x 2 block
  if (threadIdx.x == 0) {
    if (n >= 2) {
      if ((n - 2) % G == b) {
        const DF* c = cols + (int64_t)((n - 2) / G) * n;
        d[n - 2] = df_to_double(c[n - 2]);
        e[n - 2] = df_to_double(c[n - 1]);
      }
      if ((n - 1) % G == b) d[n - 1] = df_to_double(cols[(int64_t)((n - 1) / G) * n + n - 1]);
    } else if (b == 0) {
      d[0] = df_to_double(cols[0]);
    }
  }
}

// ---------------------------------------------------------------------------- 2. eigenvalues
// lam_asc[i] (ascending), one half-warp per eigenvalue: 16 Sturm counts per step shrink the
// bracket 17-fold, down to a relative width 2 eps (so that eigenvalues far below eps ||T|| stay
// apart and their twisted vectors differ).  The count of eigenvalues below x is the number of sign
// changes of the leading principal minors p_j(x) = (d_j - x) p_{j-1} - e_{j-1}^2 p_{j-2}
// (Sturm sequence), evaluated without divisions and kept in range by exact power-of-two
// rescaling; a minor that is exactly zero takes the sign opposite to its predecessor and a
// magnitude 2^-200 times it (a negative pivot, as in LAPACK's pivmin rule).  GB300 retires about
// two FP64 operations per cycle and SM, so a step of the recurrence costs three of them (the
// shift, the product with e^2, the FMA) and nothing else: the sign and zero tests work on the bit
// patterns in the integer pipes without branches, and the range test runs every fourth step.
// T and x are scaled by a power of two to ||T|| ~ 1 (the counts do not change), and off-diagonals
// with |e_j| <= eps ||T|| are dropped (the matrix splits there; a perturbation below the rounding
// of T), so that e_j^2 >= eps^2: a step then changes the larger of the last two minors by at most
// a factor 2^3 up, or eps^2 down (a cancellation), and rescaling whenever that exponent leaves
// [-400, 400] keeps four steps inside the normal range.  Sixteen counts per eigenvalue balance
// the FP64 throughput against the latency of the recurrence's chain.
constexpr long long kAbsBits = 0x7fffffffffffffffLL;
constexpr long long kSignBit = (long long)0x8000000000000000ULL;

__device__ __forceinline__ void sturm_step(double dj, double e2j, double x, double& pm, double& pc, long long& bc,
                                           int& c) {
  double pn = fma(dj - x, pc, -e2j * pm);
  long long bn = __double_as_longlong(pn);
  // exact zero: -sign(pc) 2^-200 |pc| (clamped to the normal range)
  const long long zr = max((bc & kAbsBits) - (200LL << 52), 1LL << 52) | (~bc & kSignBit);
  bn = (bn & kAbsBits) == 0 ? zr : bn;
  c += (int)((unsigned long long)(bn ^ bc) >> 63);
  pm = pc;
  pc = __longlong_as_double(bn);
  bc = bn;
}

__device__ __forceinline__ int sturm_count(const double* __restrict__ d, const double* __restrict__ e2, int n,
                                           double x) {
  double pm = 1.0, pc = d[0] - x;
  long long bc = __double_as_longlong(pc);
  if ((bc & kAbsBits) == 0) {
    pc = -0x1p-200;
    bc = __double_as_longlong(pc);
  }
  int c = (int)((unsigned long long)bc >> 63);
  int j = 1;
  for (; j + 4 <= n; j += 4) {
    sturm_step(d[j], e2[j - 1], x, pm, pc, bc, c);
    sturm_step(d[j + 1], e2[j], x, pm, pc, bc, c);
    sturm_step(d[j + 2], e2[j + 1], x, pm, pc, bc, c);
    sturm_step(d[j + 3], e2[j + 2], x, pm, pc, bc, c);
    const int ex = max((int)((bc >> 52) & 0x7ff), (int)((__double_as_longlong(pm) >> 52) & 0x7ff));
    if (ex > 1023 + 400 || ex < 1023 - 400) {            // rescale both terms by 2^(1023 - ex)
      const double sc = __longlong_as_double((long long)(2046 - ex) << 52);
      pc *= sc;
      pm *= sc;
      bc = __double_as_longlong(pc);
    }
  }
  for (; j < n; ++j) sturm_step(d[j], e2[j - 1], x, pm, pc, bc, c);
  return c;
}

constexpr int kSectLanes = 16;
constexpr int kSectThreads = 32;   // two eigenvalues per block (an FP64 instruction costs the same
                                   // with 16 active lanes as with 32: measured)
constexpr unsigned kSectMask = kSectThreads == 32 ? 0xffffffffu : (1u << kSectThreads) - 1u;

__global__ void __launch_bounds__(kSectThreads) k_multisect(const double* __restrict__ d, const double* __restrict__ e,
                                                           int n, double* __restrict__ lam_asc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* ds = reinterpret_cast<double*>(smem_raw);   // [n]
  double* e2 = ds + n;                                // [n]
  double lo = DBL_MAX, hi = -DBL_MAX;                 // Gershgorin interval, once per block
  for (int j = threadIdx.x; j < n; j += kSectThreads) {
    const double dj = d[j];
    const double ej = j + 1 < n ? fabs(e[j]) : 0.0, ejm = j > 0 ? fabs(e[j - 1]) : 0.0;
    lo = fmin(lo, dj - ej - ejm);
    hi = fmax(hi, dj + ej + ejm);
  }
#pragma unroll
  for (int o = kSectThreads / 2; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(kSectMask, lo, o));
    hi = fmax(hi, __shfl_xor_sync(kSectMask, hi, o));
  }
  const double tn = fmax(fmax(fabs(lo), fabs(hi)), DBL_MIN);
  const double tsc = __longlong_as_double((long long)(2046 - (int)((__double_as_longlong(tn) >> 52) & 0x7ff)) << 52);
  for (int j = threadIdx.x; j < n; j += kSectThreads) {   // scaled copy, ||T|| in [1, 2)
    ds[j] = d[j] * tsc;
    const double ej = j + 1 < n ? fabs(e[j]) : 0.0;
    e2[j] = ej > DBL_EPSILON * tn ? (ej * tsc) * (ej * tsc) : 0.0;
  }
  __syncwarp(kSectMask);
  const int sl = threadIdx.x & (kSectLanes - 1), half = (threadIdx.x >> 4) & 1;
  const unsigned hmask = 0xffffu << (16 * half);
  const int i = (blockIdx.x * kSectThreads + threadIdx.x) / kSectLanes;
  if (i >= n) return;                                 // whole half-warps leave together
  const double span = fmax(hi - lo, fmax(fabs(hi), fabs(lo)));
  const double atol = 2.0 * DBL_EPSILON * span + DBL_MIN;
  // width floor eps^2 ||T||: eigenvalues far below the rounding of T stay apart (relative width
  // 2 eps above it) without the bisection running on to the underflow threshold
  const double wfloor = DBL_EPSILON * DBL_EPSILON * span + 4.0 * DBL_MIN;
  double a = lo - atol, b = hi + atol;
  for (int it = 0; it < 160; ++it) {
    if (b - a <= fmax(2.0 * DBL_EPSILON * fmax(fabs(a), fabs(b)), wfloor)) break;
    const double h = (b - a) * (1.0 / (kSectLanes + 1));
    const double x = a + h * (sl + 1);
    const int c = sturm_count(ds, e2, n, x * tsc);
    const unsigned mask = (__ballot_sync(hmask, c > i) >> (16 * half)) & 0xffffu;
    if (mask == 0u) {
      a = a + h * kSectLanes;
    } else {
      const int l = __ffs(mask) - 1;
      const double nb = a + h * (l + 1);
      a = l == 0 ? a : a + h * l;
      b = nb;
    }
  }
  if (sl == 0) lam_asc[i] = 0.5 * (a + b);
}

// Double-float multisection (FP32 contexts): the count of eigenvalues below x as the number of
// negative pivots of T - x I = L D L^T, q_j = (d_j - x) - e_{j-1}^2 / q_{j-1} with |q_j| kept
// above FP32's safe minimum times max(1, max e^2) (LAPACK's pivmin rule, so e^2 / q stays
// finite), each division an FP32 reciprocal refined by one double-float step.  No rescaling is
// needed, the chain is tens of FP32-pipe cycles per step instead of the FP64 pipe's issue-bound
// three operations, and each lane evaluates two points (64 per eigenvalue and step).
namespace {

__device__ __forceinline__ float rcp_approx(float x) {   // one MUFU operation, ~1 ulp
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// a / b: q0 = a_hi / b_hi from the approximate reciprocal, then q = q0 + (a - q0 b) / b_hi; the
// correction brings ~2^-22 to ~2^-44
__device__ __forceinline__ DF df_divq(DF a, DF b) {
  const float rb = rcp_approx(b.hi);
  const float q0 = a.hi * rb;
  const float p = q0 * b.hi;
  const float pe = fmaf(q0, b.hi, -p);
  float r = (a.hi - p) - pe;
  r = fmaf(-q0, b.lo, r + a.lo);
  const float q1 = r * rb;
  const float hi = q0 + q1;
  return DF{hi, q1 - (hi - q0)};
}

__device__ __forceinline__ void pivot_step(DF dj, DF e2, DF x, DF& q, int& c, float pivmin) {
  DF t = df_add(dj, DF{-x.hi, -x.lo});
  t = df_add(t, df_neg(df_divq(e2, q)));
  if (fabsf(t.hi) < pivmin) t = DF{-pivmin, 0.f};
  c += t.hi < 0.f;
  q = t;
}

}  // namespace

__global__ void __launch_bounds__(32) k_multisect_df(const double* __restrict__ d, const double* __restrict__ e, int n,
                                                     double* __restrict__ lam_asc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DF* ds = reinterpret_cast<DF*>(smem_raw);           // [n], scaled
  DF* e2 = ds + n;                                    // [n], scaled squares
  double lo = DBL_MAX, hi = -DBL_MAX;
  for (int j = threadIdx.x; j < n; j += 32) {
    const double dj = d[j];
    const double ej = j + 1 < n ? fabs(e[j]) : 0.0, ejm = j > 0 ? fabs(e[j - 1]) : 0.0;
    lo = fmin(lo, dj - ej - ejm);
    hi = fmax(hi, dj + ej + ejm);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
  }
  const double tn = fmax(fmax(fabs(lo), fabs(hi)), DBL_MIN);
  const double tsc = __longlong_as_double((long long)(2046 - (int)((__double_as_longlong(tn) >> 52) & 0x7ff)) << 52);
  float e2max = 0.f;
  for (int j = threadIdx.x; j < n; j += 32) {           // scaled copy, ||T|| in [1, 2)
    DF a, b;
    split_df(d[j] * tsc, a.hi, a.lo);
    const double ej = j + 1 < n ? e[j] * tsc : 0.0;
    split_df(ej * ej, b.hi, b.lo);
    ds[j] = a;
    e2[j] = b;
    e2max = fmaxf(e2max, b.hi);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e2max = fmaxf(e2max, __shfl_xor_sync(0xffffffffu, e2max, o));
  __syncwarp();
  const float pivmin = FLT_MIN * fmaxf(1.f, e2max);
  const int i = blockIdx.x;                           // one eigenvalue per warp
  const int lane = threadIdx.x;
  const double span = fmax(hi - lo, fmax(fabs(hi), fabs(lo)));
  const double atol = 2.0 * DBL_EPSILON * span + DBL_MIN;
  const double wfloor = DBL_EPSILON * DBL_EPSILON * span + 4.0 * DBL_MIN;
  // Points per step: 32 P, two per lane (a warp's step then issues about as many instructions as
  // the dependent chain of one point takes cycles).  While the bracket spans more than a factor of
  // 4 (or holds zero) the points are spaced evenly in s(x) = sign(x) log2(1 + |x| / wfloor), i.e.
  // geometrically above wfloor: a small eigenvalue of a wide spectrum is then located to a factor
  // of ~3 in one step instead of shrinking the bracket by 32 P per step from ||T|| down.  Any
  // increasing points refine the bracket (the counts are monotone in x); FP32 placement suffices
  // while the bracket is that wide.
  constexpr int P = 2;
  constexpr int M = 32 * P;
  const double inv_wf = 1.0 / wfloor;
  double a = lo - atol, b = hi + atol;
  for (int it = 0; it < 160; ++it) {
    if (b - a <= fmax(2.0 * DBL_EPSILON * fmax(fabs(a), fabs(b)), wfloor)) break;
    const bool wide = (a <= 0.0 && b >= 0.0) || (b - a > 4.0 * fmin(fabs(a), fabs(b)));
    float sa = 0.f, ds_ = 0.f;
    if (wide) {
      sa = copysignf(log2f(1.f + (float)(fabs(a) * inv_wf)), (float)a);
      const float sb = copysignf(log2f(1.f + (float)(fabs(b) * inv_wf)), (float)b);
      ds_ = (sb - sa) * (1.f / (M + 1));
    }
    const double h = (b - a) * (1.0 / (M + 1));
    double xv[P];
    DF x[P], q[P];
    int cnt[P];
#pragma unroll
    for (int u = 0; u < P; ++u) {                     // point u * 32 + lane (ascending in the warp's order)
      const int k = u * 32 + lane + 1;
      if (wide) {
        const float sk = sa + ds_ * k;
        xv[u] = copysign(wfloor * (double)(exp2f(fabsf(sk)) - 1.f), (double)sk);
      } else {
        xv[u] = a + h * k;
      }
      split_df(xv[u] * tsc, x[u].hi, x[u].lo);
      q[u] = df_add(ds[0], df_neg(x[u]));
      if (fabsf(q[u].hi) < pivmin) q[u] = DF{-pivmin, 0.f};
      cnt[u] = q[u].hi < 0.f;
    }
    for (int j = 1; j < n; ++j) {
      const DF dj = ds[j], ej = e2[j - 1];
#pragma unroll
      for (int u = 0; u < P; ++u) pivot_step(dj, ej, x[u], q[u], cnt[u], pivmin);
    }
    // first of the points (ascending) whose count exceeds i: lambda_i lies between it and the point
    // before it (or a); none: above the last point
    int pt = M;
#pragma unroll
    for (int u = P - 1; u >= 0; --u) {
      const unsigned m = __ballot_sync(0xffffffffu, cnt[u] > i);
      if (m) pt = u * 32 + __ffs(m) - 1;
    }
    const double x_last = __shfl_sync(0xffffffffu, xv[P - 1], 31);
    if (pt == M) {
      a = fmax(a, x_last);
    } else {
      const int u = pt >> 5, l = pt & 31;
      double xb = xv[0], xa = xv[0];
#pragma unroll
      for (int w = 0; w < P; ++w) {
        const double vb = __shfl_sync(0xffffffffu, xv[w], l);
        const double va = __shfl_sync(0xffffffffu, xv[w], (l + 31) & 31);
        if (w == u) xb = vb;
        if (w == (l == 0 ? u - 1 : u)) xa = va;
      }
      if (pt > 0) a = fmax(a, xa);
      b = fmin(b, xb);
    }
  }
  if (lane == 0) lam_asc[i] = 0.5 * (a + b);
}

// ---------------------------------------------------------------------------- 3. eigenvectors of T
// Z[:, i] = unit eigenvector of T for lam_asc[i] by the twisted factorization, one thread per
// eigenvalue.  The recurrences are chains of dependent FP64 divisions and products, so their
// operands sit in shared memory: d, e for the block and, per thread, D+ (kept in z), L+ and U-,
// interleaved by thread ([j][kTwThreads]).  Lp, Um: global scratch (n x n) for the variant that
// keeps the per-thread arrays in global memory when they do not fit.
constexpr int kTwThreads = 4;

template <bool SMEM>
__global__ void __launch_bounds__(kTwThreads) k_twisted(const double* __restrict__ d, const double* __restrict__ e,
                                                       int n, const double* __restrict__ lam_asc,
                                                       double* __restrict__ Z, double* __restrict__ Lp,
                                                       double* __restrict__ Um) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sd = reinterpret_cast<double*>(smem_raw);   // [n]
  double* se = sd + n;                                // [n]
  for (int j = threadIdx.x; j < n; j += kTwThreads) {
    sd[j] = d[j];
    se[j] = j + 1 < n ? e[j] : 0.0;
  }
  __syncthreads();
  const int t = threadIdx.x;
  const int i = blockIdx.x * kTwThreads + t;
  if (i >= n) return;
  // per-thread arrays: element j of thread t at base[j * st + t]
  const int64_t st = SMEM ? kTwThreads : 1;
  double* zb = SMEM ? se + n : Z + (int64_t)i * n;
  double* Lb = SMEM ? zb + (int64_t)n * kTwThreads : Lp + (int64_t)i * n;
  double* Ub = SMEM ? Lb + (int64_t)n * kTwThreads : Um + (int64_t)i * n;
  const int off = SMEM ? t : 0;
  auto Z_ = [&](int j) -> double& { return zb[(int64_t)j * st + off]; };
  auto L_ = [&](int j) -> double& { return Lb[(int64_t)j * st + off]; };
  auto U_ = [&](int j) -> double& { return Ub[(int64_t)j * st + off]; };
  double emax = 0.0;
  for (int j = 0; j + 1 < n; ++j) emax = fmax(emax, se[j] * se[j]);
  const double pivmin = DBL_MIN * fmax(1.0, emax);
  const double lam = lam_asc[i];
  // forward: D+_j and L+_j = e_j / D+_j; D+ kept in z (overwritten later)
  double dp = sd[0] - lam;
  Z_(0) = dp;
  for (int j = 1; j < n; ++j) {
    if (fabs(dp) < pivmin) dp = dp < 0.0 ? -pivmin : pivmin;
    const double l = se[j - 1] / dp;
    L_(j - 1) = l;
    dp = sd[j] - lam - l * se[j - 1];
    Z_(j) = dp;
  }
  // backward: D-_j and U-_j = e_{j-1} / D-_j; twist index from gamma_r = D+_r + D-_r - (d_r - lam)
  double dm = sd[n - 1] - lam;
  int r = n - 1;
  double best = fabs(Z_(n - 1));   // gamma_{n-1} = D+_{n-1}
  for (int j = n - 1; j >= 1; --j) {
    if (fabs(dm) < pivmin) dm = dm < 0.0 ? -pivmin : pivmin;
    const double u = se[j - 1] / dm;
    U_(j) = u;
    dm = sd[j - 1] - lam - u * se[j - 1];
    const double g = fabs(Z_(j - 1) + dm - (sd[j - 1] - lam));
    if (g < best) {
      best = g;
      r = j - 1;
    }
  }
  // z_r = 1, z_j = -L+_j z_{j+1} (j < r), z_j = -U-_j z_{j-1} (j > r)
  Z_(r) = 1.0;
  double nrm = 1.0;
  for (int j = r - 1; j >= 0; --j) {
    Z_(j) = -L_(j) * Z_(j + 1);
    nrm += Z_(j) * Z_(j);
  }
  for (int j = r + 1; j < n; ++j) {
    Z_(j) = -U_(j) * Z_(j - 1);
    nrm += Z_(j) * Z_(j);
  }
  const double sc = 1.0 / sqrt(nrm);
  double* zo = Z + (int64_t)i * n;
  for (int j = 0; j < n; ++j) zo[j] = Z_(j) * sc;
}

size_t twisted_smem(int n) { return (size_t)(2 + 3 * kTwThreads) * n * sizeof(double); }

// The same twisted factorization in double-float arithmetic on the FP32 pipes (FP32 contexts,
// whose Nystrom core is FP64-accurate to ~2^-48 anyway): each FP64 division of the recurrences
// (~560 cycles of dependent FP64 latency on GB300) becomes an FP32 reciprocal and one
// double-float correction step (tens of cycles).  The pivot floor is FP32's safe minimum
// FLT_MIN max(1, max e_j^2), so that e_j / pivot stays finite, as in the FP64 form with DBL_MIN.
// Per-thread arrays in shared memory as pairs: [j][kTwThreads] of (hi, lo).
namespace {

__device__ __forceinline__ DF df_mul2(DF a, DF b) { return df_mul(a, b.hi, b.lo); }

// a / b: q0 = a_hi / b_hi in FP32, then q = q0 + (a - q0 b) / b_hi
__device__ __forceinline__ DF df_div(DF a, DF b) {
  const float rb = rcp_approx(b.hi);
  const float q0 = a.hi * rb;
  const float p = q0 * b.hi;
  const float pe = fmaf(q0, b.hi, -p);                 // q0 b_hi = p + pe exactly
  float r = (a.hi - p) - pe;
  r = fmaf(-q0, b.lo, r + a.lo);
  const float q1 = r * rb;
  const float hi = q0 + q1;
  return DF{hi, q1 - (hi - q0)};
}

__device__ __forceinline__ float df_abs_hi(DF a) { return fabsf(a.hi); }

}  // namespace

__global__ void __launch_bounds__(kTwThreads) k_twisted_df(const double* __restrict__ d, const double* __restrict__ e,
                                                          int n, const double* __restrict__ lam_asc,
                                                          double* __restrict__ Z) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DF* sd = reinterpret_cast<DF*>(smem_raw);           // [n]
  DF* se = sd + n;                                    // [n]
  DF* zb = se + n;                                    // [n][kTwThreads]
  DF* Lb = zb + (int64_t)n * kTwThreads;
  DF* Ub = Lb + (int64_t)n * kTwThreads;
  float emax = 0.f;
  for (int j = threadIdx.x; j < n; j += kTwThreads) {
    DF a, b;
    split_df(d[j], a.hi, a.lo);
    split_df(j + 1 < n ? e[j] : 0.0, b.hi, b.lo);
    sd[j] = a;
    se[j] = b;
  }
  __syncthreads();
  const int t = threadIdx.x;
  const int i = blockIdx.x * kTwThreads + t;
  if (i >= n) return;
  for (int j = 0; j + 1 < n; ++j) emax = fmaxf(emax, se[j].hi * se[j].hi);
  const float pivmin = FLT_MIN * fmaxf(1.f, emax);
  auto Z_ = [&](int j) -> DF& { return zb[(int64_t)j * kTwThreads + t]; };
  auto L_ = [&](int j) -> DF& { return Lb[(int64_t)j * kTwThreads + t]; };
  auto U_ = [&](int j) -> DF& { return Ub[(int64_t)j * kTwThreads + t]; };
  DF lam;
  split_df(lam_asc[i], lam.hi, lam.lo);
  const DF nlam = df_neg(lam);
  // forward: D+_j and L+_j = e_j / D+_j; D+ kept in z
  DF dp = df_add(sd[0], nlam);
  Z_(0) = dp;
  for (int j = 1; j < n; ++j) {
    if (df_abs_hi(dp) < pivmin) dp = DF{dp.hi < 0.f ? -pivmin : pivmin, 0.f};
    const DF l = df_div(se[j - 1], dp);
    L_(j - 1) = l;
    dp = df_add(df_add(sd[j], nlam), df_neg(df_mul2(l, se[j - 1])));
    Z_(j) = dp;
  }
  // backward: D-_j and U-_j = e_{j-1} / D-_j; twist index from gamma_r = D+_r + D-_r - (d_r - lam)
  DF dm = df_add(sd[n - 1], nlam);
  int r = n - 1;
  float best = df_abs_hi(Z_(n - 1));
  for (int j = n - 1; j >= 1; --j) {
    if (df_abs_hi(dm) < pivmin) dm = DF{dm.hi < 0.f ? -pivmin : pivmin, 0.f};
    const DF u = df_div(se[j - 1], dm);
    U_(j) = u;
    const DF dl = df_add(sd[j - 1], nlam);
    dm = df_add(dl, df_neg(df_mul2(u, se[j - 1])));
    const float g = fabsf(df_add(df_add(Z_(j - 1), dm), df_neg(dl)).hi);
    if (g < best) {
      best = g;
      r = j - 1;
    }
  }
  // z_r = 1, z_j = -L+_j z_{j+1} (j < r), z_j = -U-_j z_{j-1} (j > r)
  Z_(r) = DF{1.f, 0.f};
  DF nrm{1.f, 0.f};
  for (int j = r - 1; j >= 0; --j) {
    const DF zj = df_neg(df_mul2(L_(j), Z_(j + 1)));
    Z_(j) = zj;
    nrm = df_add(nrm, df_mul2(zj, zj));
  }
  for (int j = r + 1; j < n; ++j) {
    const DF zj = df_neg(df_mul2(U_(j), Z_(j - 1)));
    Z_(j) = zj;
    nrm = df_add(nrm, df_mul2(zj, zj));
  }
  const double sc = 1.0 / sqrt(df_to_double(nrm));
  double* zo = Z + (int64_t)i * n;
  for (int j = 0; j < n; ++j) zo[j] = df_to_double(Z_(j)) * sc;
}


// ---------------------------------------------------------------------------- 4. back-transform
// V[:, c] = H_0 H_1 ... H_{n-3} Z[:, c_src] with c_src = n-1-c (descending eigenvalues); one warp
// per column, the column held in shared memory, H_k = I - tau_k v_k v_k^T acting on rows k+1..n-1.
__global__ void __launch_bounds__(128) k_backtransform(const double* __restrict__ Z, int n,
                                                       const double* __restrict__ tau, const double* __restrict__ Vh,
                                                       double* __restrict__ V) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double* out = reinterpret_cast<double*>(smem_raw) + (int64_t)warp * n;
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (c >= n) return;
  const double* src = Z + (int64_t)(n - 1 - c) * n;
  for (int i = lane; i < n; i += 32) out[i] = src[i];
  __syncwarp();
  for (int k = n - 3; k >= 0; --k) {
    const double tk = tau[k];
    if (tk == 0.0) continue;
    const int m = n - k - 1;
    const double* vk = Vh + (int64_t)k * n;
    double s = 0.0;
    for (int i = lane; i < m; i += 32) s += vk[i] * out[k + 1 + i];
    s = wsum_d(s) * tk;
    for (int i = lane; i < m; i += 32) out[k + 1 + i] -= s * vk[i];
    __syncwarp();
  }
  double* dst = V + (int64_t)c * n;
  for (int i = lane; i < n; i += 32) dst[i] = out[i];
}

// Double-float form for n <= 32 NQ + 1: one warp per two columns, the columns in shared memory as
// packed f32x2 pairs (column 0 and column 1 in the two lanes of each register), so that one
// instruction serves both columns; the next reflector's entries are fetched into registers while
// the current one is applied.  Per reflector: s = tau v^T x (double-float products and sums, a
// warp butterfly), x -= s v, each updated entry renormalised.  ~2^-48 relative error per
// operation, on the FP32 pipes instead of GB300's narrow FP64 pipe.
namespace {

__device__ __forceinline__ DF2 df2_add(DF2 a, DF2 b) {
  const f2x s = add2(a.hi, b.hi);
  const f2x z = sub2(s, a.hi);
  f2x e = add2(sub2(a.hi, sub2(s, z)), sub2(b.hi, z));
  e = add2(e, add2(a.lo, b.lo));
  const f2x hi = add2(s, e);
  return DF2{hi, sub2(e, sub2(hi, s))};
}

// acc += (ah + al)(bh + bl), lane-wise
__device__ __forceinline__ void df2_mac4(DF2& acc, f2x ah, f2x al, f2x bh, f2x bl) {
  const f2x pn = mul2(ah ^ 0x8000000080000000ull, bh);
  f2x pe = fma2(ah, bh, pn);
  pe = fma2(ah, bl, pe);
  pe = fma2(al, bh, pe);
  const f2x t = sub2(acc.hi, pn);
  const f2x z = sub2(t, acc.hi);
  const f2x er = sub2(sub2(acc.hi, sub2(t, z)), add2(pn, z));
  acc.hi = t;
  acc.lo = add2(add2(acc.lo, pe), er);
}

}  // namespace

template <int NQ>
__global__ void __launch_bounds__(32) k_backtransform_df(const double* __restrict__ Z, int n,
                                                         const double* __restrict__ tau, const float* __restrict__ VH,
                                                         const float* __restrict__ VL, double* __restrict__ V) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  f2x* xh = reinterpret_cast<f2x*>(smem_raw);          // [n]: high words of the two columns
  f2x* xl = xh + n;                                    // [n]: low words
  const int lane = threadIdx.x;
  const int c0 = 2 * blockIdx.x;                       // output columns c0 and c0 + 1
  const bool two = c0 + 1 < n;
  const double* s0 = Z + (int64_t)(n - 1 - c0) * n;
  const double* s1 = two ? Z + (int64_t)(n - 2 - c0) * n : s0;
  for (int i = lane; i < n; i += 32) {
    float h0, l0, h1, l1;
    split_df(s0[i], h0, l0);
    split_df(two ? s1[i] : 0.0, h1, l1);
    xh[i] = pk2(h0, h1);
    xl[i] = pk2(l0, l1);
  }
  __syncwarp();
  float nh[NQ], nl[NQ];
  double ntk = 0.0;
  auto fetch = [&](int k) {
    const int m = n - k - 1;
    const float* vkh = VH + (int64_t)k * n;
    const float* vkl = VL + (int64_t)k * n;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const bool in = lane + 32 * q < m;
      nh[q] = in ? vkh[lane + 32 * q] : 0.f;
      nl[q] = in ? vkl[lane + 32 * q] : 0.f;
    }
    ntk = tau[k];
  };
  if (n >= 3) fetch(n - 3);
  for (int k = n - 3; k >= 0; --k) {
    const int m = n - k - 1;
    float vh[NQ], vl[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      vh[q] = nh[q];
      vl[q] = nl[q];
    }
    const double tk = ntk;
    if (k > 0) fetch(k - 1);
    if (tk == 0.0) continue;                           // uniform over the warp
    DF2 a4[4] = {{0ull, 0ull}, {0ull, 0ull}, {0ull, 0ull}, {0ull, 0ull}};   // four independent chains
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int i = lane + 32 * q;
      if (i < m) df2_mac4(a4[q & 3], xh[k + 1 + i], xl[k + 1 + i], pk2(vh[q], vh[q]), pk2(vl[q], vl[q]));
    }
    DF2 acc = df2_add(df2_add(a4[0], a4[1]), df2_add(a4[2], a4[3]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      acc = df2_add(acc, DF2{__shfl_xor_sync(0xffffffffu, acc.hi, o), __shfl_xor_sync(0xffffffffu, acc.lo, o)});
    // s = -tau acc
    float th, tl;
    split_df(-tk, th, tl);
    DF2 sv;
    {
      const f2x bth = pk2(th, th), btl = pk2(tl, tl);
      const f2x p = mul2(acc.hi, bth);
      f2x pe = fma2(acc.hi, bth, p ^ 0x8000000080000000ull);
      pe = fma2(acc.hi, btl, pe);
      pe = fma2(acc.lo, bth, pe);
      const f2x hi = add2(p, pe);
      sv = DF2{hi, sub2(pe, sub2(hi, p))};
    }
    // x += s v, renormalised
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int i = lane + 32 * q;
      if (i < m) {
        DF2 x{xh[k + 1 + i], xl[k + 1 + i]};
        df2_mac4(x, sv.hi, sv.lo, pk2(vh[q], vh[q]), pk2(vl[q], vl[q]));
        const f2x hi = add2(x.hi, x.lo);
        xh[k + 1 + i] = hi;
        xl[k + 1 + i] = sub2(x.lo, sub2(hi, x.hi));
      }
    }
    __syncwarp();
  }
  for (int i = lane; i < n; i += 32) {
    float h0, h1, l0, l1;
    upk2(xh[i], h0, h1);
    upk2(xl[i], l0, l1);
    V[(int64_t)c0 * n + i] = f32_to_f64(h0) + f32_to_f64(l0);
    if (two) V[(int64_t)(c0 + 1) * n + i] = f32_to_f64(h1) + f32_to_f64(l1);
  }
}

// Blocked form of the double-float back-transform: the reflectors in blocks of kWy (block b:
// k = kWy b .. min(kWy b + kWy - 1, n - 3)), each block's product H_k0 H_k0+1 ... H_k1 written in
// the compact WY form I - Y T Y^T (Schreiber and Van Loan, "A storage-efficient WY representation
// for products of Householder transformations", SIAM J. Sci. Stat. Comput. 10 (1989)): column j
// of Y is the reflector vector of H_k0+j (zero above row k0 + j + 1), T is upper triangular with
// T_jj = tau_j and T[0:j, j] = -tau_j T[0:j, 0:j] (Y[:, 0:j]^T y_j).  A block then acts on a set of
// columns X as X -= Y (T (Y^T X)): two small matrix products per kWy reflectors, where the
// one-reflector form runs kWy dependent warp-wide dot products and updates.
constexpr int kWy = 32;
constexpr int kWyCols = 4;          // eigenvector columns per CTA of the apply kernel
constexpr int kWyThreads = 512;
constexpr int kWyTRows = 256;       // rows of Y per shared-memory chunk in k_wy_t

// Rows [r0, r0 + rows) of block b's Y into Yc[rr][0..kWy) (row stride kWy + 1): entry (r, j) =
// v_{k0+j}[r - k0 - j - 1] for r > k0 + j and j < nbk, else zero (so that the products need no
// masks).  Consecutive threads read consecutive entries of one reflector; each thread issues eight
// loads before it stores any (the L2 latency once per eight entries, not per entry).
__device__ __forceinline__ void wy_load_rows(const float* __restrict__ VH, const float* __restrict__ VL, int n, int k0,
                                             int nbk, int r0, int rows, DF* __restrict__ Yc, int tid, int nthr) {
  constexpr int U = 8;
  const int total = rows * kWy;
  for (int base = tid; base < total; base += U * nthr) {
    float h[U], l[U];
    int dst[U];
#pragma unroll
    for (int t = 0; t < U; ++t) {
      const int idx = base + t * nthr;
      h[t] = 0.f;
      l[t] = 0.f;
      dst[t] = -1;
      if (idx < total) {
        const int j = idx / rows, rr = idx - j * rows, r = r0 + rr;
        dst[t] = rr * (kWy + 1) + j;
        if (j < nbk && r > k0 + j) {
          const int64_t o = (int64_t)(k0 + j) * n + (r - k0 - j - 1);
          h[t] = VH[o];
          l[t] = VL[o];
        }
      }
    }
#pragma unroll
    for (int t = 0; t < U; ++t)
      if (dst[t] >= 0) Yc[dst[t]] = DF{h[t], l[t]};
  }
}

// T of every block: TH / TL [b][kWy][kWy] row-major (zero below the diagonal and past the block's
// last reflector).  One CTA per block: S = Y^T Y (strict upper triangle, a thread per entry over
// shared-memory chunks of Y's rows), then the recurrence for T by one warp (lane = row of T).
__global__ void __launch_bounds__(512) k_wy_t(int n, const double* __restrict__ tau, const float* __restrict__ VH,
                                              const float* __restrict__ VL, float* __restrict__ TH,
                                              float* __restrict__ TL) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DF* Yc = reinterpret_cast<DF*>(smem_raw);                 // [kWyTRows][kWy + 1]
  __shared__ DF S[kWy][kWy + 1];
  __shared__ DF T[kWy][kWy + 1];
  const int b = blockIdx.x, k0 = b * kWy;
  const int nbk = min(kWy, n - 2 - k0);
  const int tid = threadIdx.x, lane = tid & 31;
  // entry pi = j (j - 1) / 2 + i of the strict upper triangle (i < j): consecutive threads share j
  const int npair = nbk * (nbk - 1) / 2;
  int pj = 1, pii = tid;
  while (pii >= pj) {
    pii -= pj;
    ++pj;
  }
  const bool has = tid < npair;
  DF a0{0.f, 0.f}, a1{0.f, 0.f};
  for (int r0 = k0 + 1; r0 < n; r0 += kWyTRows) {
    const int rows = min(kWyTRows, n - r0);
    __syncthreads();
    wy_load_rows(VH, VL, n, k0, nbk, r0, rows, Yc, tid, blockDim.x);
    __syncthreads();
    if (has) {
      int rr = 0;
      for (; rr + 1 < rows; rr += 2) {
        const DF x0 = Yc[rr * (kWy + 1) + pii], y0 = Yc[rr * (kWy + 1) + pj];
        const DF x1 = Yc[(rr + 1) * (kWy + 1) + pii], y1 = Yc[(rr + 1) * (kWy + 1) + pj];
        df_add_prod2(a0, x0.hi, x0.lo, y0.hi, y0.lo);
        df_add_prod2(a1, x1.hi, x1.lo, y1.hi, y1.lo);
      }
      if (rr < rows) {
        const DF x0 = Yc[rr * (kWy + 1) + pii], y0 = Yc[rr * (kWy + 1) + pj];
        df_add_prod2(a0, x0.hi, x0.lo, y0.hi, y0.lo);
      }
    }
  }
  if (has) S[pii][pj] = df_add(a0, a1);
  __syncthreads();
  if (tid < 32) {
    for (int c = 0; c < kWy; ++c) T[lane][c] = DF{0.f, 0.f};
    __syncwarp();
    for (int j = 0; j < nbk; ++j) {
      float th, tl;
      split_df(tau[k0 + j], th, tl);
      DF v{th, tl};
      if (lane < j) {
        // -tau_j sum over l in [lane, j) of T[lane][l] S[l][j], four chains
        DF c4[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
        for (int l = lane; l < j; ++l) df_add_prod2(c4[(l - lane) & 3], T[lane][l].hi, T[lane][l].lo, S[l][j].hi, S[l][j].lo);
        v = df_mul(df_add(df_add(c4[0], c4[1]), df_add(c4[2], c4[3])), -th, -tl);
      }
      __syncwarp();
      if (lane <= j) T[lane][j] = v;
      __syncwarp();
    }
    float* th_b = TH + (int64_t)b * kWy * kWy;
    float* tl_b = TL + (int64_t)b * kWy * kWy;
    for (int r = 0; r < kWy; ++r) {
      th_b[r * kWy + lane] = T[r][lane].hi;
      tl_b[r * kWy + lane] = T[r][lane].lo;
    }
  }
}

// Rows of Y a k_wy_apply chunk holds for n (shared memory: X, the chunk, the static arrays).
__host__ __device__ inline int wy_apply_rows(int n) {
  const int avail = (200 * 1024 - n * kWyCols * 8 - 11 * 1024) / ((kWy + 1) * 8);
  return avail < n ? avail : n;
}

// V[:, c] = H_0 H_1 ... H_{n-3} Z[:, n-1-c] for the CTA's kWyCols columns c (X in shared memory as
// double-float, row-major [n][kWyCols]), the blocks applied from the last to the first.  Per
// block, over shared-memory chunks of Y's rows: W = Y^T X (four threads per entry of W, each over
// every fourth row of the chunk), W2 = T W, X -= Y W2 (a thread per row); a chunk holding all the
// block's rows serves both products.
__global__ void __launch_bounds__(kWyThreads) k_wy_apply(const double* __restrict__ Z, int n,
                                                         const float* __restrict__ VH, const float* __restrict__ VL,
                                                         const float* __restrict__ TH, const float* __restrict__ TL,
                                                         double* __restrict__ V) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  DF* X = reinterpret_cast<DF*>(smem_raw);                  // [n][kWyCols]
  DF* Yc = X + (int64_t)n * kWyCols;                        // [RC][kWy + 1]
  __shared__ DF W[kWy][kWyCols], W2[kWy][kWyCols];
  __shared__ DF Ts[kWy][kWy + 1];
  const int RC = wy_apply_rows(n);
  const int tid = threadIdx.x;
  const int c0 = blockIdx.x * kWyCols;
  for (int idx = tid; idx < n * kWyCols; idx += kWyThreads) {
    const int q = idx / n, r = idx - q * n;
    float h = 0.f, l = 0.f;
    if (c0 + q < n) split_df(Z[(int64_t)(n - 1 - c0 - q) * n + r], h, l);
    X[r * kWyCols + q] = DF{h, l};
  }
  const int nblk = n >= 3 ? (n - 2 + kWy - 1) / kWy : 0;
  // W entry (j, q) of this thread and its row residue
  const int wo = tid >> 2, wj = wo / kWyCols, wq = wo % kWyCols, ws = tid & 3;
  for (int b = nblk - 1; b >= 0; --b) {
    const int k0 = b * kWy, nbk = min(kWy, n - 2 - k0);
    const int rbeg = k0 + 1, nrow = n - rbeg;
    const bool one_chunk = nrow <= RC;
    __syncthreads();                                          // X of the previous block, Yc free
    for (int idx = tid; idx < kWy * kWy; idx += kWyThreads)
      Ts[idx / kWy][idx % kWy] = DF{TH[(int64_t)b * kWy * kWy + idx], TL[(int64_t)b * kWy * kWy + idx]};
    DF acc{0.f, 0.f}, acc2{0.f, 0.f};
    for (int r0 = rbeg; r0 < n; r0 += RC) {
      const int rows = min(RC, n - r0);
      if (r0 > rbeg) __syncthreads();
      wy_load_rows(VH, VL, n, k0, nbk, r0, rows, Yc, tid, kWyThreads);
      __syncthreads();
      if (wo < kWy * kWyCols) {
        int rr = ws;
        for (; rr + 4 < rows; rr += 8) {
          const DF y0 = Yc[rr * (kWy + 1) + wj], x0 = X[(r0 + rr) * kWyCols + wq];
          const DF y1 = Yc[(rr + 4) * (kWy + 1) + wj], x1 = X[(r0 + rr + 4) * kWyCols + wq];
          df_add_prod2(acc, y0.hi, y0.lo, x0.hi, x0.lo);
          df_add_prod2(acc2, y1.hi, y1.lo, x1.hi, x1.lo);
        }
        if (rr < rows) {
          const DF y0 = Yc[rr * (kWy + 1) + wj], x0 = X[(r0 + rr) * kWyCols + wq];
          df_add_prod2(acc, y0.hi, y0.lo, x0.hi, x0.lo);
        }
      }
    }
    // the four threads of an entry are lanes 4o .. 4o + 3 of one warp
    acc = df_add(acc, acc2);
    acc = df_add(acc, shfl_xor_df(acc, 1));
    acc = df_add(acc, shfl_xor_df(acc, 2));
    if (ws == 0 && wo < kWy * kWyCols) W[wj][wq] = acc;
    __syncthreads();
    // W2 = T W (T upper triangular)
    if (tid < kWy * kWyCols) {
      const int j = tid / kWyCols, q = tid % kWyCols;
      DF a0{0.f, 0.f}, a1{0.f, 0.f};
      int i = j;
      for (; i + 1 < nbk; i += 2) {
        df_add_prod2(a0, Ts[j][i].hi, Ts[j][i].lo, W[i][q].hi, W[i][q].lo);
        df_add_prod2(a1, Ts[j][i + 1].hi, Ts[j][i + 1].lo, W[i + 1][q].hi, W[i + 1][q].lo);
      }
      if (i < nbk) df_add_prod2(a0, Ts[j][i].hi, Ts[j][i].lo, W[i][q].hi, W[i][q].lo);
      W2[j][q] = j < nbk ? df_add(a0, a1) : DF{0.f, 0.f};
    }
    __syncthreads();
    // X[r] -= Y[r] W2 (Y's zeros above each reflector's start make the row's sum run over all kWy)
    for (int r0 = rbeg; r0 < n; r0 += RC) {
      const int rows = min(RC, n - r0);
      if (!one_chunk) {
        __syncthreads();
        wy_load_rows(VH, VL, n, k0, nbk, r0, rows, Yc, tid, kWyThreads);
        __syncthreads();
      }
      for (int rr = tid; rr < rows; rr += kWyThreads) {
        DF s4[kWyCols];
#pragma unroll
        for (int q = 0; q < kWyCols; ++q) s4[q] = DF{0.f, 0.f};
        const DF* yr = Yc + rr * (kWy + 1);
        for (int j = 0; j < nbk; ++j) {
          const DF y = yr[j];
#pragma unroll
          for (int q = 0; q < kWyCols; ++q) df_add_prod2(s4[q], y.hi, y.lo, W2[j][q].hi, W2[j][q].lo);
        }
        DF* xr = X + (int64_t)(r0 + rr) * kWyCols;
#pragma unroll
        for (int q = 0; q < kWyCols; ++q) xr[q] = df_add(xr[q], df_neg(s4[q]));
      }
    }
  }
  __syncthreads();
  for (int idx = tid; idx < n * kWyCols; idx += kWyThreads) {
    const int q = idx / n, r = idx - q * n;
    if (c0 + q < n) V[(int64_t)(c0 + q) * n + r] = df_to_double(X[r * kWyCols + q]);
  }
}

__global__ void k_add_diag(double* __restrict__ G, int n, double sh) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) G[i + (int64_t)i * n] += sh;
}

// Re-orthonormalization helpers.  G holds V^T V in its lower triangle (i >= j).  k_ns_finish
// writes the Newton-Schulz correction D = (I - G) / 2 to the whole matrix and, per block, the sum
// of (G - I)^2 over the entries it visits (off-diagonal entries counted twice), in a fixed order.
constexpr int kNsBlocks = 64;

__global__ void __launch_bounds__(256) k_ns_finish(double* __restrict__ G, int n, double* __restrict__ part) {
  __shared__ double red[8];
  const int64_t total = (int64_t)n * n;
  double acc = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    if (i < j) continue;
    const double dev = i == j ? G[e] - 1.0 : G[e];
    acc += (i == j ? 1.0 : 2.0) * dev * dev;
    const double dv = -0.5 * dev;                    // exact: G = I - 2 D is recoverable
    G[e] = dv;
    if (i != j) G[j + (int64_t)i * n] = dv;
  }
  acc = wsum_d(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

// G = I - 2 D (undoes k_ns_finish exactly, for the CholeskyQR fallback)
__global__ void k_ns_undo(double* __restrict__ G, int n) {
  const int64_t total = (int64_t)n * n;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    G[e] = (i == j ? 1.0 : 0.0) - 2.0 * G[e];
  }
}

// V += sum_z part[z] (the K slices of V D, summed in slice order)
__global__ void k_add_slices(double* __restrict__ V, const double* __restrict__ part, int nz, int64_t stride,
                             int64_t total) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    double t = part[e];
    for (int z = 1; z < nz; ++z) t += part[(int64_t)z * stride + e];
    V[e] += t;
  }
}

__global__ void k_reverse(const double* __restrict__ lam_asc, int n, double* __restrict__ lam_desc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) lam_desc[i] = lam_asc[n - 1 - i];
}

int coop_grid(const void* kernel, int threads, size_t smem) {
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem);
  return std::max(1, std::min(per, 2)) * nsm;
}

}  // namespace

constexpr int kEigSlices = 4;     // at most this many K slices in the n x n x n products below

size_t sym_eig_workspace_doubles(int n) {
  const size_t nt = (size_t)(n - 1 + 31) / 32 + 1;
  return (4 + kEigSlices) * (size_t)n * n + nt * 32 * nt + nt * nt + 12 * (size_t)n + 1024;
}

namespace {

// K slices for an n x n x n double-float product: enough blocks to cover the SMs (these products
// are small), slices at least 64 deep.
int eig_slices(int n, bool lower) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int64_t tm = (n + 127) / 128, tn = (n + 63) / 64;
  int64_t tiles = tm * tn;
  if (lower) {
    tiles = 0;
    for (int64_t a = 0; a < tm; ++a) tiles += std::min<int64_t>(tn, 2 * (a + 1));
  }
  int ns = 1;
  while (ns < kEigSlices && tiles * ns < nsm && n / (ns + 1) >= 64) ++ns;
  return ns;
}

int slice_count(int64_t K, int ns) {
  const int64_t kps = ns > 1 ? ((K + ns - 1) / ns + 15) / 16 * 16 : std::max<int64_t>(K, 1);
  return (int)((K + kps - 1) / kps);
}

// G (lower triangle) = V^T V, FP64-accurate on the FP32 pipes
void gram_lower(const double* V, int n, double* G, double* part, cudaStream_t s) {
  GemmDfArgs<double, double> g;
  g.M = n; g.N = n; g.K = n;
  g.A = V; g.sam = n; g.sak = 1;
  g.B = V; g.sbk = 1; g.sbn = n;
  g.scm = 1; g.scn = n;
  g.lower = 1;
  g.nsplit = eig_slices(n, true);
  const int nz = slice_count(n, g.nsplit);
  if (nz > 1) {
    g.out64 = part; g.split_stride = (int64_t)n * n;
    launch_gemm_df<double, double>(g, s);
    launch_sum_splits(part, nz, (int64_t)n * n, (int64_t)n * n, G, s);
  } else {
    g.out64 = G;
    launch_gemm_df<double, double>(g, s);
  }
}

}  // namespace

// Eigen-decomposition of the symmetric n x n matrix S (column-major): lam_desc (n, decreasing),
// V (n x n, column j = eigenvector of lam_desc[j]).  S is left untouched; ws holds
// sym_eig_workspace_doubles(n) doubles.
cudaError_t launch_sym_eig(const double* S, int n, double* lam_desc, double* V, double* ws, int* status,
                           cudaStream_t s, bool df_recurrences) {
  const size_t nn = (size_t)n * n;
  const size_t nt = (size_t)(n - 1 + 31) / 32 + 1;
  double* A = ws;                    // copy of S, reduced in place; later the L+ scratch
  double* Vh = A + nn;               // Householder vectors
  double* Z = Vh + nn;               // eigenvectors of T; later the CholeskyQR Gram matrix
  double* LU = Z + nn;               // U- scratch; later the row-major Cholesky factor
  double* ppart = LU + nn;
  double* tdot = ppart + nt * 32 * nt;
  double* d = tdot + nt * nt;
  double* e = d + n;
  double* tau = e + n;
  double* lam_asc = tau + n;
  double* vbuf = lam_asc + n;        // distributed reduction: v, p (2 n each), flags (n words),
  double* pbuf = vbuf + 2 * n;       // per-block partials (<= 2 x 1024 doubles with the tail)
  unsigned* flags = reinterpret_cast<unsigned*>(pbuf + 2 * n);
  double* redb = pbuf + 2 * n + n;
  cudaError_t err = cudaMemcpyAsync(A, S, nn * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (err != cudaSuccess) return err;
  cudaMemsetAsync(tau, 0, n * sizeof(double), s);
  cudaMemsetAsync(e, 0, n * sizeof(double), s);
  int nsm = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int gdist = std::max(1, std::min(nsm, 512));     // 2 gdist partials fit the tail of the workspace
  const size_t dist_smem = (size_t)((n + gdist - 1) / gdist + 2) * n * sizeof(double);
  if (dist_smem <= 200 * 1024) {
    // A stays in shared memory across the grid, one block per SM
    // double-float columns (8 bytes per entry, as FP64) in FP32 contexts
    const void* kern = df_recurrences ? (const void*)k_tridiag_dist_df : (const void*)k_tridiag_dist;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dist_smem);
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 256, dist_smem);
    if (per < 1) return cudaErrorCooperativeLaunchTooLarge;
    int nn_ = n;
    const double* Ac = A;
    cudaMemsetAsync(flags, 0, (size_t)n * sizeof(unsigned), s);
    void* args[] = {&Ac, &nn_, &d, &e, &tau, &Vh, &vbuf, &pbuf, &redb, &flags, &status};
    note_launch();
    err = cudaLaunchCooperativeKernel(kern, gdist, 256, args, dist_smem, s);
    if (err != cudaSuccess) return err;
  } else {
    const size_t smem = (size_t)n * sizeof(double);
    cudaFuncSetAttribute((const void*)k_tridiag, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int blocks = coop_grid((const void*)k_tridiag, 256, smem);
    int nn_ = n;
    void* args[] = {&A, &nn_, &d, &e, &tau, &Vh, &ppart, &tdot};
    note_launch();
    err = cudaLaunchCooperativeKernel((const void*)k_tridiag, blocks, 256, args, smem, s);
    if (err != cudaSuccess) return err;
  }
  if (df_recurrences) {
    const size_t smem = 2 * (size_t)n * sizeof(DF);
    cudaFuncSetAttribute((const void*)k_multisect_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_multisect_df<<<n, 32, smem, s>>>(d, e, n, lam_asc);
    note_launch();
  } else {
    const size_t smem = 2 * (size_t)n * sizeof(double);
    cudaFuncSetAttribute((const void*)k_multisect, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_multisect<<<(n * kSectLanes + kSectThreads - 1) / kSectThreads, kSectThreads, smem, s>>>(d, e, n, lam_asc);
    note_launch();
  }
  {
    const size_t smem = twisted_smem(n);
    const unsigned grid = (unsigned)((n + kTwThreads - 1) / kTwThreads);
    if (df_recurrences && smem <= 200 * 1024) {
      cudaFuncSetAttribute((const void*)k_twisted_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_twisted_df<<<grid, kTwThreads, smem, s>>>(d, e, n, lam_asc, Z);
    } else if (smem <= 200 * 1024) {
      cudaFuncSetAttribute((const void*)k_twisted<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_twisted<true><<<grid, kTwThreads, smem, s>>>(d, e, n, lam_asc, Z, A, LU);
    } else {
      const size_t smem2 = 2 * (size_t)n * sizeof(double);
      cudaFuncSetAttribute((const void*)k_twisted<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
      k_twisted<false><<<grid, kTwThreads, smem2, s>>>(d, e, n, lam_asc, Z, A, LU);
    }
    note_launch();
  }
  if (df_recurrences && n >= 64 && wy_apply_rows(n) >= 64) {
    // blocked (compact WY) form: the reflectors as double-float pairs once (into the free L+ / U-
    // scratch A), the blocks' T factors into the free LU scratch (nblk kWy^2 pairs <= n^2 doubles)
    float* VH = reinterpret_cast<float*>(A);
    float* VL = VH + nn;
    launch_split_df(Vh, VH, VL, (int64_t)nn, (int64_t)nn, s);
    const int nblk = (n - 2 + kWy - 1) / kWy;
    float* TH = reinterpret_cast<float*>(LU);
    float* TL = TH + (size_t)nblk * kWy * kWy;
    const int tsm = kWyTRows * (kWy + 1) * (int)sizeof(DF);
    cudaFuncSetAttribute((const void*)k_wy_t, cudaFuncAttributeMaxDynamicSharedMemorySize, tsm);
    k_wy_t<<<nblk, 512, tsm, s>>>(n, tau, VH, VL, TH, TL);
    note_launch();
    const size_t smem = ((size_t)n * kWyCols + (size_t)wy_apply_rows(n) * (kWy + 1)) * sizeof(DF);
    cudaFuncSetAttribute((const void*)k_wy_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_wy_apply<<<(n + kWyCols - 1) / kWyCols, kWyThreads, smem, s>>>(Z, n, VH, VL, TH, TL, V);
    note_launch();
  } else if (df_recurrences && n <= 32 * 32 + 1) {   // the longest reflector, n - 1 entries, within 32 NQ lanes
    // the reflectors as double-float pairs once (into the free L+ / U- scratch), so that no warp
    // converts FP64 in its loop
    float* VH = reinterpret_cast<float*>(A);
    float* VL = VH + nn;
    launch_split_df(Vh, VH, VL, (int64_t)nn, (int64_t)nn, s);
    const size_t smem = 2 * (size_t)n * sizeof(f2x);
    if (n <= 32 * 16 + 1) {
      k_backtransform_df<16><<<(n + 1) / 2, 32, smem, s>>>(Z, n, tau, VH, VL, V);
    } else {
      k_backtransform_df<32><<<(n + 1) / 2, 32, smem, s>>>(Z, n, tau, VH, VL, V);
    }
    note_launch();
  } else {
    const size_t smem = 4 * (size_t)n * sizeof(double);
    cudaFuncSetAttribute((const void*)k_backtransform, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_backtransform<<<(n * 32 + 127) / 128, 128, smem, s>>>(Z, n, tau, Vh, V); note_launch();
  }
  k_reverse<<<(n + 255) / 256, 256, 0, s>>>(lam_asc, n, lam_desc); note_launch();
  // Re-orthonormalization of V.  G = V^T V = I + E; while ||E||_F <= 1/2, Newton-Schulz steps
  // V <- V (3 I - G) / 2 = V + V D, D = (I - G) / 2, converge to the orthonormal polar factor of V
  // (each singular value s of V goes to s (3 - s^2) / 2, so a deviation e of s^2 from 1 becomes
  // -(3/4) e^2 + e^3 / 4).  Each vector moves by half its overlaps with the others, so vectors of
  // well-separated eigenvalues, already orthogonal to eps ||T|| / gap, stay put.  Otherwise (nearly
  // equal vectors from eigenvalues below the core's rounding) shifted CholeskyQR and two plain
  // passes turn them into an orthonormal basis of their joint invariant subspace.
  double* G = Z;
  double* part = ws + (sym_eig_workspace_doubles(n) - (size_t)kEigSlices * nn);
  gram_lower(V, n, G, part, s);
  k_ns_finish<<<kNsBlocks, 256, 0, s>>>(G, n, redb); note_launch();
  launch_sum_partials(redb, kNsBlocks, 1.0, redb + kNsBlocks, s);
  double fro2 = 0.0;
  err = cudaMemcpyAsync(&fro2, redb + kNsBlocks, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  if (err != cudaSuccess) return err;
  const double fro = sqrt(fro2);
  if (fro <= 0.5) {
    int steps = 0;
    for (double ev = fro; ev > 4e-16 && steps < 8; ev = 0.75 * ev * ev * (1.0 + ev / 3.0)) ++steps;
    for (int it = 0; it < steps; ++it) {
      if (it > 0) {
        gram_lower(V, n, G, part, s);
        k_ns_finish<<<kNsBlocks, 256, 0, s>>>(G, n, redb); note_launch();
      }
      GemmDfArgs<double, double> g;                   // part = V D (K slices)
      g.M = n; g.N = n; g.K = n;
      g.A = V; g.sam = 1; g.sak = n;
      g.B = G; g.sbk = 1; g.sbn = n;
      g.scm = 1; g.scn = n;
      g.nsplit = eig_slices(n, false);
      const int nz = slice_count(n, g.nsplit);
      g.out64 = part; g.split_stride = (int64_t)n * n;
      launch_gemm_df<double, double>(g, s);
      const int blocks = (int)std::min<int64_t>(((int64_t)n * n + 255) / 256, 4 * 152);
      k_add_slices<<<blocks, 256, 0, s>>>(V, part, nz, (int64_t)n * n, (int64_t)n * n); note_launch();
    }
    return cudaGetLastError();
  }
  {
    const int blocks = (int)std::min<int64_t>(((int64_t)n * n + 255) / 256, 4 * 152);
    k_ns_undo<<<blocks, 256, 0, s>>>(G, n); note_launch();
  }
  for (int pass = 0; pass < 3; ++pass) {
    if (pass > 0) {
      gram_lower(V, n, G, part, s);
      launch_mirror_lower(G, n, s);
    } else {
      // shift 1e-12 n: far above the rounding of the Gram matrix of n unit columns (~eps n), far
      // below the unit diagonal
      k_add_diag<<<(n + 255) / 256, 256, 0, s>>>(G, n, 1e-12 * n); note_launch();
    }
    err = launch_cholesky(G, n, status, s);
    if (err != cudaSuccess) return err;
    launch_trsm_lt<double>(V, n, n, n, G, LU, s);
  }
  return cudaGetLastError();
}

}  // namespace ngd
