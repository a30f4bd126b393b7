// FP64 symmetric eigen-decomposition of the l x l Nystrom core S = B^T B (App. A: the thin SVD
// of B, read as eig(B^T B) and U = B V Sigma^{-1}).
//
// GB300 has few FP64 units per SM (~8 flop/clk) and a grid-wide barrier costs ~1.2 us, so the
// solver keeps the number of dependent steps and the FP64 work per SM low:
//   1. Householder tridiagonalization S = Q T Q^T in one cooperative kernel: per column two
//      grid barriers; the symmetric matrix-vector product and the rank-2 update are spread
//      over 32 x 32 tiles of the trailing block on all SMs (deterministic partial sums).
//   2. Eigenvalues of T by multisection (one warp per eigenvalue, 32 Sturm counts per step).
//   3. Eigenvectors of T by one twisted factorization per eigenvalue (one thread each):
//      T - lambda I = L+ D+ L+^T = U- D- U-^T, twist index r = argmin |gamma_r|,
//      gamma_r = D+_r + D-_r - (d_r - lambda), z_r = 1 and the two bidiagonal recurrences.
//   4. V = Q Z by applying the reflectors to the columns of Z (one warp per column, no barrier).
//   5. V is re-orthonormalised by shifted CholeskyQR followed by two plain CholeskyQR passes
//      (Fukaya, Kannan, Nakatsukasa, Yamamoto, Yanagisawa, SIAM J. Sci. Comput. 2020), columns in
//      decreasing eigenvalue order.  Twisted vectors of well-separated eigenvalues are already
//      orthogonal to eps ||T|| / gap; eigenvalues closer than the rounding of S (the noise floor
//      of the Nystrom core) can give (nearly) equal vectors, which the shifted pass turns into an
//      orthonormal basis of their joint invariant subspace.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>

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

// ---------------------------------------------------------------------------- 2. eigenvalues
// lam_asc[i] (ascending), one warp per eigenvalue: 32 Sturm counts (number of negative LDL^T
// pivots of T - x I) per step shrink the bracket 33-fold, down to a relative width 2 eps (so
// that eigenvalues far below eps ||T|| stay apart and their twisted vectors differ).
__global__ void k_multisect(const double* __restrict__ d, const double* __restrict__ e, int n,
                            double* __restrict__ lam_asc) {
  const int lane = threadIdx.x & 31;
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= n) return;
  double lo = DBL_MAX, hi = -DBL_MAX, emax = 0.0;
  for (int j = 0; j < n; ++j) {       // Gershgorin interval
    const double ej = j + 1 < n ? fabs(e[j]) : 0.0, ejm = j > 0 ? fabs(e[j - 1]) : 0.0;
    lo = fmin(lo, d[j] - ej - ejm);
    hi = fmax(hi, d[j] + ej + ejm);
    emax = fmax(emax, ej * ej);
  }
  const double pivmin = DBL_MIN * fmax(1.0, emax);
  const double span = fmax(hi - lo, fmax(fabs(hi), fabs(lo)));
  const double atol = 2.0 * DBL_EPSILON * span;
  double a = lo - atol - pivmin, b = hi + atol + pivmin;
  for (int it = 0; it < 96; ++it) {
    if (b - a <= 2.0 * DBL_EPSILON * fmax(fabs(a), fabs(b)) + 4.0 * pivmin) break;
    const double h = (b - a) / 33.0;
    const double x = a + h * (lane + 1);
    double q = d[0] - x;
    int c = q < 0.0;
    for (int j = 1; j < n; ++j) {
      if (fabs(q) < pivmin) q = -pivmin;
      q = d[j] - x - (e[j - 1] * e[j - 1]) / q;
      c += q < 0.0;
    }
    const unsigned mask = __ballot_sync(0xffffffffu, c > i);
    if (mask == 0u) {
      a = a + h * 32.0;
    } else {
      const int l = __ffs(mask) - 1;
      const double nb = a + h * (l + 1);
      a = l == 0 ? a : a + h * l;
      b = nb;
    }
  }
  if (lane == 0) lam_asc[i] = 0.5 * (a + b);
}

// ---------------------------------------------------------------------------- 3. eigenvectors of T
// Z[:, i] = unit eigenvector of T for lam_asc[i] by the twisted factorization; Lp, Um scratch (n x n).
__global__ void k_twisted(const double* __restrict__ d, const double* __restrict__ e, int n,
                          const double* __restrict__ lam_asc, double* __restrict__ Z, double* __restrict__ Lp,
                          double* __restrict__ Um) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double emax = 0.0;
  for (int j = 0; j + 1 < n; ++j) emax = fmax(emax, e[j] * e[j]);
  const double pivmin = DBL_MIN * fmax(1.0, emax);
  const double lam = lam_asc[i];
  double* L = Lp + (int64_t)i * n;   // L+_j, j = 0..n-2; stores D+_j in L[n-1] slot only transiently
  double* U = Um + (int64_t)i * n;   // U-_j, j = 1..n-1
  double* z = Z + (int64_t)i * n;
  // forward: D+_j and L+_j = e_j / D+_j; keep D+ in z (overwritten later)
  double dp = d[0] - lam;
  z[0] = dp;
  for (int j = 1; j < n; ++j) {
    if (fabs(dp) < pivmin) dp = dp < 0.0 ? -pivmin : pivmin;
    const double l = e[j - 1] / dp;
    L[j - 1] = l;
    dp = d[j] - lam - l * e[j - 1];
    z[j] = dp;
  }
  // backward: D-_j and U-_j = e_{j-1} / D-_j; twist index from gamma_r = D+_r + D-_r - (d_r - lam)
  double dm = d[n - 1] - lam;
  int r = n - 1;
  double best = fabs(z[n - 1]);   // gamma_{n-1} = D+_{n-1}
  for (int j = n - 1; j >= 1; --j) {
    if (fabs(dm) < pivmin) dm = dm < 0.0 ? -pivmin : pivmin;
    const double u = e[j - 1] / dm;
    U[j] = u;
    dm = d[j - 1] - lam - u * e[j - 1];
    const double g = fabs(z[j - 1] + dm - (d[j - 1] - lam));
    if (g < best) {
      best = g;
      r = j - 1;
    }
  }
  // z_r = 1, z_j = -L+_j z_{j+1} (j < r), z_j = -U-_j z_{j-1} (j > r)
  z[r] = 1.0;
  double nrm = 1.0;
  for (int j = r - 1; j >= 0; --j) {
    z[j] = -L[j] * z[j + 1];
    nrm += z[j] * z[j];
  }
  for (int j = r + 1; j < n; ++j) {
    z[j] = -U[j] * z[j - 1];
    nrm += z[j] * z[j];
  }
  const double s = 1.0 / sqrt(nrm);
  for (int j = 0; j < n; ++j) z[j] *= s;
}

// ---------------------------------------------------------------------------- 4. back-transform
// V[:, c] = H_0 H_1 ... H_{n-3} Z[:, c_src] with c_src = n-1-c (descending eigenvalues); one warp
// per column, H_k = I - tau_k v_k v_k^T acting on rows k+1..n-1.
__global__ void k_backtransform(const double* __restrict__ Z, int n, const double* __restrict__ tau,
                                const double* __restrict__ Vh, double* __restrict__ V) {
  const int lane = threadIdx.x & 31;
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (c >= n) return;
  double* out = V + (int64_t)c * n;
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
}

__global__ void k_add_diag(double* __restrict__ G, int n, double sh) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) G[i + (int64_t)i * n] += sh;
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

size_t sym_eig_workspace_doubles(int n) {
  const size_t nt = (size_t)(n - 1 + 31) / 32 + 1;
  return 4 * (size_t)n * n + nt * 32 * nt + nt * nt + 6 * (size_t)n;
}

// Eigen-decomposition of the symmetric n x n matrix S (column-major): lam_desc (n, decreasing),
// V (n x n, column j = eigenvector of lam_desc[j]).  S is left untouched; ws holds
// sym_eig_workspace_doubles(n) doubles.
cudaError_t launch_sym_eig(const double* S, int n, double* lam_desc, double* V, double* ws, int* status,
                           cudaStream_t s) {
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
  cudaError_t err = cudaMemcpyAsync(A, S, nn * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (err != cudaSuccess) return err;
  cudaMemsetAsync(tau, 0, n * sizeof(double), s);
  cudaMemsetAsync(e, 0, n * sizeof(double), s);
  {
    const size_t smem = (size_t)n * sizeof(double);
    cudaFuncSetAttribute((const void*)k_tridiag, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int blocks = coop_grid((const void*)k_tridiag, 256, smem);
    int nn_ = n;
    void* args[] = {&A, &nn_, &d, &e, &tau, &Vh, &ppart, &tdot};
    note_launch();
    err = cudaLaunchCooperativeKernel((const void*)k_tridiag, blocks, 256, args, smem, s);
    if (err != cudaSuccess) return err;
  }
  k_multisect<<<(n * 32 + 255) / 256, 256, 0, s>>>(d, e, n, lam_asc); note_launch();
  k_twisted<<<(n + 127) / 128, 128, 0, s>>>(d, e, n, lam_asc, Z, A, LU); note_launch();
  k_backtransform<<<(n * 32 + 127) / 128, 128, 0, s>>>(Z, n, tau, Vh, V); note_launch();
  k_reverse<<<(n + 255) / 256, 256, 0, s>>>(lam_asc, n, lam_desc); note_launch();
  // shifted CholeskyQR, then CholeskyQR2: G = V^T V (+ s I), G = L L^T, V <- V L^{-T}
  for (int pass = 0; pass < 3; ++pass) {
    GemmArgs<double> g;
    g.M = n; g.N = n; g.K = n;
    g.A = V; g.sam = n; g.sak = 1;
    g.B = V; g.sbk = 1; g.sbn = n;
    g.outT = Z; g.scm = 1; g.scn = n;
    launch_gemm<double>(g, s);
    launch_symmetrize(Z, n, s);
    // shift 1e-12 n on the first pass: far above the rounding of the Gram matrix of n unit columns
    // (~eps n), far below the unit diagonal
    if (pass == 0) {
      k_add_diag<<<(n + 255) / 256, 256, 0, s>>>(Z, n, 1e-12 * n); note_launch();
    }
    err = launch_cholesky(Z, n, status, s);
    if (err != cudaSuccess) return err;
    launch_trsm_lt<double>(V, n, n, n, Z, LU, lam_asc, s);
  }
  return cudaGetLastError();
}

}  // namespace ngd
