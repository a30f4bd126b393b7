// Declarations of the dense kernels in linalg.cu and the double-float GEMM in gemm_df.cu.
#pragma once

#include "ngd_internal.cuh"

namespace ngd {

constexpr int kRedBlocks = 1024;   // maximum number of per-block partials of one reduction

// Device-resident scalars of one preconditioned-CG solve.
struct PcgScalars {
  double rz, pq, alpha, beta, rn2, gn2, rtol2;
  int done, iters, maxit, status, cur_iter;
  unsigned int counter;
};

// Strided SIMT GEMM C(m,n) = sum_k A(m,k) B(k,n) (see k_gemm).
template <typename T> struct GemmArgs {
  int64_t M = 0, N = 0, K = 0;
  const T* A = nullptr; int64_t sam = 0, sak = 0;
  const T* B = nullptr; int64_t sbk = 0, sbn = 0;
  int nsplit = 1;                     // K slices (FP64 partial per slice into out64)
  double* out64 = nullptr; int64_t split_stride = 0;
  T* outT = nullptr;
  int64_t scm = 0, scn = 0;
  const double* rowscale = nullptr;   // per-m factor (nullable)
  const double* colscale = nullptr;   // per-n factor (nullable)
  int accumulate = 0;                 // out64 += result instead of out64 = result (nsplit must be 1)
};

// FP64-accurate (double-float) SIMT GEMM, operands float or double, FP64 or FP32 output.
template <typename TA, typename TB> struct GemmDfArgs {
  int64_t M = 0, N = 0, K = 0;
  const TA* A = nullptr; int64_t sam = 0, sak = 0;
  const TB* B = nullptr; int64_t sbk = 0, sbn = 0;
  int nsplit = 1;
  double* out64 = nullptr; int64_t split_stride = 0;
  float* out32 = nullptr;
  int64_t scm = 0, scn = 0;
  const double* rowscale = nullptr;
  const double* colscale = nullptr;
  int accumulate = 0;
  int lower = 0;     // write only out[m][n] with n <= m (M x N square output); skip tiles above
};
template <typename TA, typename TB> void launch_gemm_df(const GemmDfArgs<TA, TB>& g, cudaStream_t s);
// K slices that fill the GPU's block slots most evenly for an M x N double-float GEMM (lower:
// only the lower-triangle tiles of a square output run)
int gemm_df_splits(int64_t M, int64_t N, int64_t K, bool lower = false);

// sampling test matrix (column selection with probabilities proportional to diag G)
template <typename T>
int launch_gram_diag(const T* J, int64_t ldJ, int64_t nrows, int64_t p, const double* w, double* part, int64_t ldp,
                     int max_splits, int accumulate, cudaStream_t s);
void launch_sample_indices(const double* d, int64_t p, int ell, uint64_t seed, uint64_t step,
                           unsigned long long* keys, int* idx, int* status, cudaStream_t s);
template <typename T> void launch_selection_omega(T* Om, int64_t ld, const int* idx, int ell, cudaStream_t s);
template <typename T, typename TO>
void launch_gather_cols(const T* J, int64_t ldJ, int64_t N, const int* idx, int ell, const double* w, TO* Zw,
                        cudaStream_t s);
// RPCholesky (block variant) and the power method
void launch_philox_column(double* v, int64_t p, uint32_t word, uint64_t seed, uint64_t step, cudaStream_t s);
void launch_scale_rsqrt(const double* src, const double* ss, double* dst, int64_t n, cudaStream_t s);
void launch_rpchol_pivots(const double* d, int64_t p, int b, int rnd, uint64_t seed, uint64_t step, int* piv,
                          int* sel, int* nsel, cudaStream_t s);
void launch_gather_rows_neg(const double* F, int64_t ld, const int* sel, int nsel, int r, double* Fs, cudaStream_t s);
void launch_pivot_block(const double* C, int64_t ld, const int* sel, int nsel, double* M, cudaStream_t s);
int launch_rpchol_diag(double* d, const double* Fn, int64_t ld, int64_t p, int nsel, const int* sel, double* part,
                       cudaStream_t s);
void launch_rpchol_lambda(const double* sig2, int r, double* lam, double* inv_sigma, cudaStream_t s);
// NGD full (Alg. 2): w .* J in FP64, diagonal shift, Cholesky solve
template <typename T>
void launch_scale_rows_f64(const T* J, int64_t ld, int64_t N, const double* w, double* Z, cudaStream_t s);
void launch_add_diag_dev(double* A, int64_t n, int64_t ld, const double* shift, cudaStream_t s);
cudaError_t launch_chol_solve(const double* L, int n, int64_t ld, const double* b, double* x, double* y,
                              cudaStream_t s);
void launch_copy_diag(const double* A, int64_t n, int64_t ld, double* dg, cudaStream_t s);
void launch_restore_lower(double* A, int64_t n, int64_t ld, const double* dg, const double* shift, cudaStream_t s);
void launch_scale_scalar(double* x, double f, cudaStream_t s);
void launch_lower_to_upper(double* A, int64_t n, int64_t ld, cudaStream_t s);
// blocked Cholesky for large n; D, W: 256 x 256 doubles, T: 256 x (n - 256) doubles of scratch.
// With oz, the trailing updates run on the digit-plane tensor-core GEMM (oz_syrk_sub), otherwise
// (or where that path cannot serve) on the double-float GEMM.
struct OzSketch;
cudaError_t launch_cholesky_blocked(double* A, int64_t n, int64_t lda, int* status, double* D, double* W, double* T,
                                    cudaStream_t s, OzSketch* oz = nullptr, long long wait_cycles = 0);


void launch_sum_partials(const double* part, int n, double scale, double* out, cudaStream_t s);
template <typename T> void launch_d2t(const double* x, T* y, int64_t n, int64_t npad, cudaStream_t s);

template <typename T>
void launch_rowdot(const T* J, int64_t ldJ, int64_t nrows, const T* v, const double* w, double* t_out,
                   double* s_out, const int* done, cudaStream_t s);
int coldot_nsplit(int64_t nrows, int64_t ldJ, int vn);
template <typename T>
void launch_coldot(const T* J, int64_t ldJ, int64_t nrows, const double* s_vec, double* part, int nsplit,
                   const int* done, cudaStream_t st);
// FP32 Jacobian, FP64-accurate sums (exact FP32 products, double-float accumulation)
void launch_split_df(const double* x, float* hi, float* lo, int64_t n, int64_t npad, cudaStream_t s);
// y = x rounded to FP32 (integer conversion), n elements
void launch_f64_to_f32(const double* x, float* y, int64_t n, cudaStream_t s);
void launch_rowdot_df(const float* J, int64_t ldJ, int64_t nrows, const float* vh, const float* vl, const double* w,
                      double* t_out, double* s_out, const int* done, cudaStream_t s);
void launch_coldot_df(const float* J, int64_t ldJ, int64_t nrows, const double* s_vec, double* part, int nsplit,
                      const int* done, cudaStream_t st);
void launch_coldot_finish(const double* part, int nsplit, int64_t p, int64_t ld_part, const double* v, double mu_h,
                          const double* mu_d, double* y, int accumulate, const int* done, cudaStream_t s);

void launch_pcg_init(const double* g, double* x, double* r, int64_t n, double* part, PcgScalars* sc, cudaStream_t s);
void launch_pcg_first_dir(const double* r, const double* z, double* pv, int64_t n, double* part, PcgScalars* sc,
                          cudaStream_t s);
void launch_pcg_alpha(const double* pv, const double* q, int64_t n, double* part, PcgScalars* sc, cudaStream_t s);
void launch_pcg_update_xr(double* x, double* r, const double* pv, const double* q, int64_t n, double* part,
                          PcgScalars* sc, cudaStream_t s);
void launch_pcg_beta(const double* r, const double* z, int64_t n, double* part, PcgScalars* sc, cudaStream_t s);
void launch_pcg_update_p(double* pv, const double* z, int64_t n, PcgScalars* sc, cudaStream_t s);
void launch_axpy_to(const double* x, const double* d, double alpha, double* y, int64_t n, cudaStream_t s);
void launch_dot(const double* a, const double* b, int64_t n, double* part, double* out, cudaStream_t s);

template <typename T>
void launch_precond(const T* U, int64_t ld, int64_t p, int ell, const double* lam, double mu_h, const double* mu_d,
                    const double* v, double* z, double* w1, const int* done, cudaStream_t s);

template <typename T>
void launch_philox_omega(T* Om, int64_t ld, int64_t p, int ell, uint64_t seed, uint64_t step, cudaStream_t s);

template <typename T> void launch_gemm(const GemmArgs<T>& g, cudaStream_t s);
// FP32 GEMM of the layer products (sgemm.cu): K-slices of FP32 accumulation, FP64 slice partials
// (out64, split_stride) or one slice into outT (accumulate honoured); rowscale/colscale unused.
int sgemm_layer_slices(int64_t M, int64_t N, int64_t K);
void launch_sgemm_layer(const GemmArgs<float>& g, int nslices, cudaStream_t s);
void launch_sum_splits(const double* part, int nz, int64_t stride, int64_t n, double* out, cudaStream_t s);
template <typename T>
void launch_sum_splits_t(const double* part, int nz, int64_t stride, int64_t rows, int64_t cols, int64_t ldp, T* out,
                         int64_t ldo, cudaStream_t s);

void launch_compute_nu(const double* frob2, int mant_bits, double scale, double* nu_out, cudaStream_t s);
template <typename T>
void launch_frob2(const T* Y, int64_t ld, int64_t p, int ell, double* part, double* out, cudaStream_t s);
template <typename T>
void launch_shift_add(const T* src, const T* Om, const double* nu, T* dst, int64_t ld, int64_t p, int ell,
                      cudaStream_t s);
void launch_symmetrize(double* M, int n, cudaStream_t s);
// upper triangle = transpose of the lower one
void launch_mirror_lower(double* M, int n, cudaStream_t s);
void launch_shift_add_mixed(const double* Y, const float* Om, const double* nu, double* dst, int64_t ld, int64_t p,
                            int ell, cudaStream_t s);

template <typename T>
void launch_trsm_lt(T* X, int64_t ld, int64_t p, int n, const double* L, T* W, cudaStream_t s);
cudaError_t launch_cholesky(double* A, int n, int* status, cudaStream_t s);
// eigen.cu: FP64 symmetric eigen-decomposition (tridiagonal reduction, multisection, twisted
// factorization, back-transform, re-orthonormalization), eigenvalues decreasing.  df_recurrences:
// multisection, twisted factorization and back-transform in double-float arithmetic (~2^-48 per
// operation, for FP32 contexts whose Nystrom core carries that precision) instead of FP64.
size_t sym_eig_workspace_doubles(int n);
cudaError_t launch_sym_eig(const double* S, int n, double* lam_desc, double* V, double* ws, int* status,
                           cudaStream_t s, bool df_recurrences = false);
void launch_nystrom_lambda(const double* sig2, const double* nu, int n, double* lam, double* inv_sigma,
                           cudaStream_t s);
void launch_set_mu(const double* lam, double fixed_mu, double gamma, const double* loss, double c, double* mu,
                   cudaStream_t s);

// Whole preconditioned CG for an FP32 stored Jacobian in one cooperative kernel (pcg_fused.cu).
struct FusedPcgArgs {
  const float* J = nullptr; int64_t ldJ = 0, N = 0, p = 0;   // J: N x ldJ row-major, zero beyond column p
  const double* w = nullptr;                                 // residual weights (N)
  const float *wh = nullptr, *wl = nullptr;                  // the weights split into FP32 pairs (N)
  const float* Uh = nullptr; const float* Ul = nullptr;      // U = Uh + Ul, j-major: U[j, k] at j * ldu + k
  const double* lam = nullptr; int ell = 0, ldu = 0;         // ell = 0: no preconditioner; ldu = ell rounded
                                                             // up to a multiple of 4 (zero padding)
  const double* mu_d = nullptr; double mu_h = 0.0;           // mu from device (if set) or host
  const double* g = nullptr;                                 // right-hand side (p)
  double *x = nullptr, *r = nullptr, *z = nullptr, *pv = nullptr, *q = nullptr;   // p each
  float *vhf = nullptr, *vlf = nullptr;                      // matvec vector split into FP32 pairs (ldJ each,
                                                             // zero beyond p)
  float *yph = nullptr, *ypl = nullptr;                      // fused_pcg_blocks() x ldJ each
  double* red = nullptr;                                     // fused_pcg_blocks() x 4
  float2* w1p = nullptr;                                     // fused_pcg_blocks() x ell
  float2* w2 = nullptr;                                      // ell
  PcgScalars* sc = nullptr;                                  // rtol2, maxit in; iterations and status out
  int mode = 0;                                              // 0: PCG; 1: q = (G + mu I) pv only
  // block group of the solve in a multi-problem launch: blocks gb0 .. gb0 + gG - 1; bar: the
  // group's barrier counter (zeroed before the launch; null: the whole grid, cooperative grid
  // barrier); wait_cycles: limit of each group barrier wait
  int gb0 = 0, gG = 0;
  unsigned int* bar = nullptr;
  long long wait_cycles = 4000000000ll;
};
int fused_pcg_blocks();
int fused_pcg_slots(int64_t ldJ);
bool fused_pcg_supported(int64_t p, int64_t ldJ, int ell);
bool fused_pcg_supported_on(int64_t p, int64_t ldJ, int ell, int G);
int fused_pcg_min_blocks(int64_t p, int ell);      // fewest blocks a solve may run on
cudaError_t launch_pcg_fused(const FusedPcgArgs& a, cudaStream_t s);
// nprob solves in one cooperative launch: tab_host[j] (and its device copy tab_dev) describes
// problem j with its block group (gb0 consecutive, gG blocks, its own zeroed barrier counter bar);
// all problems share fused_pcg_slots(ldJ) rounded up to even.
cudaError_t launch_pcg_fused_multi(const FusedPcgArgs* tab_dev, const FusedPcgArgs* tab_host, int nprob,
                                   cudaStream_t s);
template <typename TU>
void launch_split_transpose_df(const TU* U, int64_t ldu, int64_t p, int ell, float* Uh, float* Ul, cudaStream_t s);

}  // namespace ngd
