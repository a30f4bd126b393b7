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
//   5. V is re-orthonormalised by CholeskyQR, columns in decreasing eigenvalue order.  Twisted
//      vectors of well-separated eigenvalues are already orthogonal to eps ||T|| / gap
//      (measured on the 5-D Poisson trajectory at ell = 500: max |V^T V - I| ~ 1e-12), and then
//      one plain pass makes them orthonormal to the working precision (CholeskyQR of a matrix with
//      condition number kappa leaves ~kappa^2 u).  Eigenvalues closer than the rounding of S (the
//      noise floor of the Nystrom core) can give (nearly) equal vectors; when max |V^T V - I|
//      exceeds 0.1 the solver takes shifted CholeskyQR followed by two plain passes instead
//      (Fukaya, Kannan, Nakatsukasa, Yamamoto, Yanagisawa, SIAM J. Sci. Comput. 2020), which
//      turns them into an orthonormal basis of their joint invariant subspace.  (A shifted first
//      pass on already orthonormal vectors would cost accuracy: it perturbs them by the shift.)
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

// Distributed variant for n small enough that each block can hold its share of A: column j
// lives in the shared memory of block j % G for the whole reduction, so per column only the
// Householder vector v and p = tau A22 v cross the grid (through L2), with two grid barriers:
//   owner of column k: v, tau (d_k, e_k)            -> barrier
//   every block: p_j = tau A[:, j] . v for its columns j > k (A symmetric), partial v . p -> barrier
//   every block: K = tau/2 v . p, w = p - K v, A[:, j] -= v w_j + w v_j for its columns;
//   the owner of column k + 1 then forms the next reflector.
// vbuf, pbuf: n doubles each; red: G doubles.
namespace {

// Householder reflector of the trailing part of column k held in col (full column, length n).
__device__ void house_from_col(const double* __restrict__ col, int n, int k, double* __restrict__ d,
                               double* __restrict__ e, double* __restrict__ tau, double* __restrict__ Vh,
                               double* __restrict__ vbuf, double* red8, double* s_bc) {
  const int m = n - k - 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double s2 = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double x = col[k + 1 + i];
    s2 += x * x;
  }
  s2 = wsum_d(s2);
  if (lane == 0) red8[warp] = s2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tsum = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tsum += red8[w];
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
      tu = 2.0 / (2.0 * (tsum + fabs(x0) * sig));
    }
    d[k] = col[k];
    e[k] = alpha;
    tau[k] = tu;
    s_bc[0] = v0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const double vi = i == 0 ? s_bc[0] : col[k + 1 + i];
    __stcg(vbuf + i, vi);
    Vh[(int64_t)k * n + i] = vi;
  }
}

}  // namespace

__global__ void __launch_bounds__(256) k_tridiag_dist(const double* __restrict__ A, int n, double* __restrict__ d,
                                                      double* __restrict__ e, double* __restrict__ tau,
                                                      double* __restrict__ Vh, double* __restrict__ vbuf,
                                                      double* __restrict__ pbuf, double* __restrict__ red) {
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
  if (n >= 3 && b == 0) house_from_col(cols, n, 0, d, e, tau, Vh, vbuf, red8, s_bc);
  grid.sync();
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;
    const double tk = __ldcg(tau + k);
    const int s_first = (k + 1 - b + G - 1) / G;          // first local slot with column j > k
    if (tk != 0.0) {                                      // uniform: every block reads the same tau
      for (int i = threadIdx.x; i < m; i += blockDim.x) vs[i] = __ldcg(vbuf + i);
      __syncthreads();
      // p_j = tau A[k+1:, j] . v for owned columns j > k, one warp per column
      double part = 0.0;
      for (int s = s_first + warp; s < ncl; s += (int)(blockDim.x >> 5)) {
        const int j = b + s * G;
        if (j >= n) break;
        const double* col = cols + (int64_t)s * n + k + 1;
        double acc = 0.0;
        for (int i = lane; i < m; i += 32) acc += col[i] * vs[i];
        const double pj = tk * wsum_d(acc);
        if (lane == 0) {
          __stcg(pbuf + (j - k - 1), pj);
          part += vs[j - k - 1] * pj;
        }
      }
      if (lane == 0) red8[warp] = part;
      __syncthreads();
      if (threadIdx.x == 0) {
        double sb = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sb += red8[w];
        __stcg(red + b, sb);
      }
      grid.sync();
      // K = tau/2 v . p (summed over blocks in block order), w = p - K v, rank-2 update
      if (warp == 0) {
        double sv = 0.0;
        for (int q = lane; q < G; q += 32) sv += __ldcg(red + q);
        sv = wsum_d(sv);
        if (lane == 0) s_bc[1] = 0.5 * tk * sv;
      }
      __syncthreads();
      const double K = s_bc[1];
      for (int i = threadIdx.x; i < m; i += blockDim.x) ws[i] = __ldcg(pbuf + i) - K * vs[i];
      __syncthreads();
      for (int s = s_first; s < ncl; ++s) {
        const int j = b + s * G;
        if (j >= n) break;
        double* col = cols + (int64_t)s * n + k + 1;
        const double wj = ws[j - k - 1], vj = vs[j - k - 1];
        for (int i = threadIdx.x; i < m; i += blockDim.x) col[i] -= vs[i] * wj + ws[i] * vj;
      }
      __syncthreads();
    } else {
      grid.sync();                                        // keep the barrier count uniform
    }
    // the owner of column k + 1 forms the next reflector from its updated column
    if (k + 3 < n && (k + 1) % G == b) house_from_col(cols + (int64_t)((k + 1) / G) * n, n, k + 1, d, e, tau, Vh, vbuf,
                                                       red8, s_bc);
    grid.sync();
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

// ---------------------------------------------------------------------------- 2. eigenvalues
// lam_asc[i] (ascending), one warp per eigenvalue: 32 Sturm counts per step shrink the bracket
// 33-fold, down to a relative width 2 eps (so that eigenvalues far below eps ||T|| stay apart
// and their twisted vectors differ).  The count of eigenvalues below x is the number of sign
// changes of the leading principal minors p_j(x) = (d_j - x) p_{j-1} - e_{j-1}^2 p_{j-2}
// (Sturm sequence), evaluated without divisions (FP64 division is slow on this GPU) and kept in
// range by exact power-of-two rescaling; a minor that is exactly zero takes the sign opposite to
// its predecessor (a negative pivot, as in LAPACK's pivmin rule).
__device__ __forceinline__ int sturm_count(const double* __restrict__ d, const double* __restrict__ e2, int n,
                                           double x) {
  double pm = 1.0, pc = d[0] - x;
  if (pc == 0.0) pc = -0x1p-1000;
  int c = pc < 0.0;
  for (int j = 1; j < n; ++j) {
    double pn = fma(d[j] - x, pc, -e2[j - 1] * pm);
    if (pn == 0.0) pn = pc < 0.0 ? 0x1p-1000 * fabs(pc) : -0x1p-1000 * fabs(pc);
    c += (pn < 0.0) != (pc < 0.0);
    pm = pc;
    pc = pn;
    const int ex = max((int)((__double_as_longlong(pc) >> 52) & 0x7ff), (int)((__double_as_longlong(pm) >> 52) & 0x7ff));
    if (ex > 1023 + 600 || ex < 1023 - 600) {            // rescale both terms by 2^(1023 - ex)
      const double sc = __longlong_as_double((long long)(2046 - ex) << 52);
      pc *= sc;
      pm *= sc;
    }
  }
  return c;
}

__global__ void k_multisect(const double* __restrict__ d, const double* __restrict__ e, int n,
                            double* __restrict__ lam_asc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* ds = reinterpret_cast<double*>(smem_raw);   // [n]
  double* e2 = ds + n;                                // [n]
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    ds[j] = d[j];
    e2[j] = j + 1 < n ? e[j] * e[j] : 0.0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= n) return;
  double lo = DBL_MAX, hi = -DBL_MAX;
  for (int j = 0; j < n; ++j) {       // Gershgorin interval
    const double ej = j + 1 < n ? fabs(e[j]) : 0.0, ejm = j > 0 ? fabs(e[j - 1]) : 0.0;
    lo = fmin(lo, ds[j] - ej - ejm);
    hi = fmax(hi, ds[j] + ej + ejm);
  }
  const double span = fmax(hi - lo, fmax(fabs(hi), fabs(lo)));
  const double atol = 2.0 * DBL_EPSILON * span + DBL_MIN;
  double a = lo - atol, b = hi + atol;
  for (int it = 0; it < 96; ++it) {
    if (b - a <= 2.0 * DBL_EPSILON * fmax(fabs(a), fabs(b)) + 4.0 * DBL_MIN) break;
    const double h = (b - a) / 33.0;
    const double x = a + h * (lane + 1);
    const int c = sturm_count(ds, e2, n, x);
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

__global__ void k_add_diag(double* __restrict__ G, int n, double sh) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) G[i + (int64_t)i * n] += sh;
}

// out = max |G - I| over the n x n matrix G (one block).
__global__ void k_max_dev_identity(const double* __restrict__ G, int n, double* __restrict__ out) {
  __shared__ double red[256];
  double m = 0.0;
  for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += blockDim.x) {
    const int i = (int)(e % n), j = (int)(e / n);
    m = fmax(m, fabs(G[e] - (i == j ? 1.0 : 0.0)));
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
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
  return 4 * (size_t)n * n + nt * 32 * nt + nt * nt + 8 * (size_t)n + 1024;
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
  double* vbuf = lam_asc + n;        // distributed reduction: v, p (n each), per-block partials (<= 1024)
  double* pbuf = vbuf + n;
  double* redb = pbuf + n;
  cudaError_t err = cudaMemcpyAsync(A, S, nn * sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (err != cudaSuccess) return err;
  cudaMemsetAsync(tau, 0, n * sizeof(double), s);
  cudaMemsetAsync(e, 0, n * sizeof(double), s);
  int nsm = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int gdist = std::max(1, std::min(nsm, 1024));
  const size_t dist_smem = (size_t)((n + gdist - 1) / gdist + 2) * n * sizeof(double);
  if (dist_smem <= 200 * 1024) {
    // A stays in shared memory across the grid, one block per SM
    cudaFuncSetAttribute((const void*)k_tridiag_dist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dist_smem);
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, (const void*)k_tridiag_dist, 256, dist_smem);
    if (per < 1) return cudaErrorCooperativeLaunchTooLarge;
    int nn_ = n;
    const double* Ac = A;
    void* args[] = {&Ac, &nn_, &d, &e, &tau, &Vh, &vbuf, &pbuf, &redb};
    note_launch();
    err = cudaLaunchCooperativeKernel((const void*)k_tridiag_dist, gdist, 256, args, dist_smem, s);
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
  {
    const size_t smem = 2 * (size_t)n * sizeof(double);
    cudaFuncSetAttribute((const void*)k_multisect, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_multisect<<<(n * 32 + 127) / 128, 128, smem, s>>>(d, e, n, lam_asc); note_launch();
  }
  k_twisted<<<(n + 7) / 8, 8, 0, s>>>(d, e, n, lam_asc, Z, A, LU); note_launch();
  {
    const size_t smem = 4 * (size_t)n * sizeof(double);
    cudaFuncSetAttribute((const void*)k_backtransform, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_backtransform<<<(n * 32 + 127) / 128, 128, smem, s>>>(Z, n, tau, Vh, V); note_launch();
  }
  k_reverse<<<(n + 255) / 256, 256, 0, s>>>(lam_asc, n, lam_desc); note_launch();
  // CholeskyQR: G = V^T V (+ s I), G = L L^T, V <- V L^{-T}; one plain pass when the twisted vectors
  // are nearly orthonormal already, else shifted CholeskyQR and two plain passes
  int passes = 1;
  for (int pass = 0; pass < passes; ++pass) {
    GemmDfArgs<double, double> g;          // FP64-accurate Gram on the FP32 pipes
    g.M = n; g.N = n; g.K = n;
    g.A = V; g.sam = n; g.sak = 1;
    g.B = V; g.sbk = 1; g.sbn = n;
    g.out64 = Z; g.scm = 1; g.scn = n;
    launch_gemm_df<double, double>(g, s);
    launch_symmetrize(Z, n, s);
    if (pass == 0) {
      k_max_dev_identity<<<1, 256, 0, s>>>(Z, n, redb); note_launch();
      double dev = 0.0;
      err = cudaMemcpyAsync(&dev, redb, sizeof(double), cudaMemcpyDeviceToHost, s);
      if (err == cudaSuccess) err = cudaStreamSynchronize(s);
      if (err != cudaSuccess) return err;
      if (!(dev <= 0.1)) {
        passes = 3;
        // shift 1e-12 n: far above the rounding of the Gram matrix of n unit columns (~eps n), far
        // below the unit diagonal
        k_add_diag<<<(n + 255) / 256, 256, 0, s>>>(Z, n, 1e-12 * n); note_launch();
      }
    }
    err = launch_cholesky(Z, n, status, s);
    if (err != cudaSuccess) return err;
    launch_trsm_lt<double>(V, n, n, n, Z, LU, s);
  }
  return cudaGetLastError();
}

}  // namespace ngd
