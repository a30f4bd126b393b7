// C ABI of libngd (include/ngd.h): context, workspace and the orchestration of the
// Nystrom-preconditioned matrix-free NGD step on one GPU.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "linalg.cuh"
#include "sketch_oz.cuh"
#include "sketch_tc.cuh"

using namespace ngd;

static std::atomic<unsigned long long> g_launches{0};
void ngd::note_launch(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }
static unsigned long long launches_now() { return g_launches.load(std::memory_order_relaxed); }

struct ngd_ctx {
  NetDesc net{};
  PointSet ps{};
  int dtype = NGD_F64;
  int gv_mode = NGD_GV_AUTO;
  size_t mem_budget = 0;
  cudaStream_t stream = nullptr;
  int64_t N = 0, p = 0, ldJ = 0, ldP = 0;
  size_t elt = 8;
  std::string err;

  bool stored_j = false;     // J (N x ldJ) is kept between matvecs
  bool tape_allowed = false; // Taylor coefficients may be stored by ngd_residual
  bool lin_valid = false;    // prep (and J when stored) match the last linearized theta
  bool tape_valid = false;   // tape matches the current prep
  bool prep_valid = false;   // prep holds the weights of a caller's theta
  uint64_t j_version = 0;    // bumped whenever the stored J changes (caches derived from J key on it)
  long long wait_cycles = 4000000000ll;  // limit of each bounded device-side wait (clock cycles)

  void* prep = nullptr;      // prepared weights of theta (working dtype)
  void* prep_t = nullptr;    // prepared tangent weights (working dtype)
  void* J = nullptr;         // N x ldJ (stored mode) or block x ldJ (matrix-free block buffer)
  int64_t jrows = 0;         // rows J can hold
  void* tape = nullptr;      // N x tape_per_point
  void* vT = nullptr;        // ldJ working-dtype vector
  double* r = nullptr;       // N residuals
  double* svec = nullptr;    // N scratch
  double* tvec = nullptr;    // N scratch
  double* part = nullptr;    // kRedBlocks partials
  double* lpart = nullptr;   // per-block loss partials of the Taylor kernels (N entries)
  double* colpart = nullptr; // coldot partials
  int colsplit = 1;
  double* scal = nullptr;    // device scalars, see kS* below
  int* status = nullptr;     // device status word
  PcgScalars* pcg = nullptr;
  double *x = nullptr, *rr = nullptr, *z = nullptr, *pv = nullptr, *q = nullptr;  // PCG vectors (p)
  double *g = nullptr, *d = nullptr, *theta_trial = nullptr;                     // step vectors (p)

  // sketch / factor workspace, grown on demand
  int ell_cap = 0;
  void *Om = nullptr, *Y = nullptr, *B = nullptr, *U = nullptr, *Lr = nullptr, *VsT = nullptr, *Zw = nullptr;
  double *M = nullptr, *A1 = nullptr, *V = nullptr, *Vs = nullptr, *sig2 = nullptr, *inv_sigma = nullptr;
  double *lam = nullptr, *dinv = nullptr, *w1 = nullptr, *gpart = nullptr, *eigws = nullptr;
  double *Y64 = nullptr, *B64 = nullptr, *Zw64 = nullptr, *U64 = nullptr;  // FP64-accurate sketch of an FP32 J
  // fused PCG (FP32 stored J): U as an FP32 pair, per-block matvec partials and reduction scratch
  float *Uh = nullptr, *Ul = nullptr, *yph = nullptr, *ypl = nullptr;
  float *vhf = nullptr, *whf = nullptr;   // split matvec vector (2 x ldJ), split weights (2 x N)
  double* fred = nullptr;
  float2 *w1p = nullptr, *w2f = nullptr;
  size_t gpart_elems = 0;
  int* perm = nullptr;
  TcSketch* tc = nullptr;
  OzSketch* oz = nullptr;    // digit planes of the FP64-accurate tensor-core sketch
  // sampling test matrix: diag G, race keys, selected columns (grown on demand)
  double* gdiag = nullptr;
  unsigned long long* samp_keys = nullptr;
  int* samp_idx = nullptr;
  int* samp_count = nullptr;
  // multi-kernel PCG: a CUDA graph of `chunk` iterations, reused while its inputs stay the same
  cudaGraphExec_t pcg_exec = nullptr;
  cudaStream_t cap_stream = nullptr;     // private stream the graph is captured on
  struct {
    const void* U; bool u_f64; int64_t ldU; const double* lam; int ell; double mu_h; const double* mu_d;
    double* x; int chunk; void* J; void* prep; bool tape;
  } pcg_key{};
  int pcg_graph_kernels = 0;
  // NGD full: the explicit Gramian (p x p, leading dimension ldG) and diag(w) J in FP64 (N x ldJ),
  // allocated on first use; for large p the scratch of the blocked Cholesky
  double* Gfull = nullptr;
  double* Zfull = nullptr;
  int64_t ldG = 0;
  double* chol_D = nullptr;
  double* chol_W = nullptr;
  double* chol_T = nullptr;

  // matrix-free VJP by layers: [pt * C + c][max_width] buffers for a chunk of rev_rows points, a
  // chunk tape when the Taylor coefficients are not stored, K-slice partials, a ones vector
  int64_t rev_rows = 0;
  void *rev_A = nullptr, *rev_X = nullptr, *rev_Xb = nullptr, *rev_tape = nullptr, *rev_ones = nullptr;

  double* h_scal = nullptr;  // pinned host scalars
  int* h_int = nullptr;
  PcgScalars* h_pcg = nullptr;
  cudaEvent_t ev[6] = {};
};

enum { kSLoss = 0, kSFrob2 = 1, kSNu = 2, kSMu = 3, kSDot = 4, kSLam1 = 5, kSTrace = 6, kSCount = 8 };
// factor attempts of ngd_step: the shift nu times 1, 8, 64, ... on NOT_SPD
constexpr int kShiftAttempts = 6;

namespace {

ngd_status set_err(ngd_ctx* c, ngd_status st, const char* fmt, const char* a = "") {
  char buf[512];
  snprintf(buf, sizeof(buf), fmt, a);
  if (c) c->err = buf;
  return st;
}

#define CK(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) return set_err(ctx, NGD_ERR_CUDA, "CUDA: %s", cudaGetErrorString(e_)); \
  } while (0)

#define TRY(call)                        \
  do {                                   \
    ngd_status s_ = (call);              \
    if (s_ != NGD_OK) return s_;         \
  } while (0)

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

template <typename P>
ngd_status dalloc(ngd_ctx* ctx, P** ptr, size_t bytes) {
  if (*ptr) {
    cudaFree(*ptr);
    *ptr = nullptr;
  }
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc((void**)ptr, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return set_err(ctx, NGD_ERR_OOM, "cudaMalloc failed: %s", cudaGetErrorString(e));
  }
  return NGD_OK;
}

ngd_status check_launch(ngd_ctx* ctx) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_err(ctx, NGD_ERR_CUDA, "kernel launch: %s", cudaGetErrorString(e));
  return NGD_OK;
}

ngd_status sync_status(ngd_ctx* ctx) {
  CK(cudaMemcpyAsync(ctx->h_int, ctx->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  const int st = ctx->h_int[0];
  // a timed-out kernel leaves its outputs unwritten: what later kernels report follows from that
  if (st & kStatTimeout)
    return set_err(ctx, NGD_ERR_TIMEOUT, (st & kStatDrain) ? "device wait timed out, and so did the drain of the work "
                                                              "already issued%s"
                                                            : "device wait timed out%s");
  if (st & kStatNotSpd) return set_err(ctx, NGD_ERR_NOT_SPD, "Nystrom core Omega^T Y_nu is not positive definite%s");
  if (st & kStatBreakdown) return set_err(ctx, NGD_ERR_BREAKDOWN, "CG breakdown: p^T (G + mu I) p <= 0%s");
  if (st & kStatNonFinite) return set_err(ctx, NGD_ERR_NONFINITE, "non-finite value in a reduction%s");
  if (st & kStatSample)
    return set_err(ctx, NGD_ERR_INVALID_ARG, "fewer positive diagonal entries of G than the sample size ell%s");
  return NGD_OK;
}

ngd_status clear_status(ngd_ctx* ctx) {
  CK(cudaMemsetAsync(ctx->status, 0, sizeof(int), ctx->stream));
  return NGD_OK;
}

// ------------------------------------------------------------------ small kernels
__global__ void k_mul(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ c, int64_t n) {
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += st) c[i] = a[i] * b[i];
}
void launch_mul(const double* a, const double* b, double* c, int64_t n, cudaStream_t s) {
  k_mul<<<(int)std::min<int64_t>((n + 255) / 256, 1024), 256, 0, s>>>(a, b, c, n); note_launch();
}

template <typename T>
__global__ void k_d2t_mat(const double* __restrict__ src, int64_t lds, T* __restrict__ dst, int64_t ldd, int64_t rows,
                          int64_t cols) {
  const int64_t n = rows * cols, st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += st) {
    const int64_t c = e / rows, r = e - c * rows;
    dst[r + c * ldd] = (T)src[r + c * lds];
  }
}

// ------------------------------------------------------------------ dtype dispatch helpers
template <typename F>
ngd_status by_dtype(ngd_ctx* ctx, F&& f) {
  if (ctx->dtype == NGD_F32) return f(float(0));
  return f(double(0));
}

ngd_status ensure_ell(ngd_ctx* ctx, int ell) {
  if (ell <= ctx->ell_cap) return NGD_OK;
  const size_t pe = (size_t)ctx->ldP * ell * ctx->elt;
  const size_t l2 = (size_t)ell * ell;
  TRY(dalloc(ctx, &ctx->Om, pe));
  TRY(dalloc(ctx, &ctx->Y, pe));
  TRY(dalloc(ctx, &ctx->B, pe));
  TRY(dalloc(ctx, &ctx->U, pe));
  TRY(dalloc(ctx, &ctx->Lr, l2 * ctx->elt));
  TRY(dalloc(ctx, &ctx->VsT, l2 * ctx->elt));
  TRY(dalloc(ctx, &ctx->Zw, (size_t)ctx->N * ell * ctx->elt));
  TRY(dalloc(ctx, &ctx->M, l2 * 8));
  TRY(dalloc(ctx, &ctx->A1, l2 * 8));
  TRY(dalloc(ctx, &ctx->V, l2 * 8));
  TRY(dalloc(ctx, &ctx->Vs, l2 * 8));
  TRY(dalloc(ctx, &ctx->sig2, ell * 8));
  TRY(dalloc(ctx, &ctx->inv_sigma, ell * 8));
  TRY(dalloc(ctx, &ctx->lam, ell * 8));
  TRY(dalloc(ctx, &ctx->dinv, ell * 8));
  TRY(dalloc(ctx, &ctx->w1, ell * 8));
  TRY(dalloc(ctx, &ctx->perm, ell * sizeof(int)));
  TRY(dalloc(ctx, &ctx->eigws, sym_eig_workspace_doubles(ell) * 8));
  if (ctx->dtype == NGD_F32) {
    TRY(dalloc(ctx, &ctx->Y64, (size_t)ctx->ldP * ell * 8));
    TRY(dalloc(ctx, &ctx->B64, (size_t)ctx->ldP * ell * 8));
    TRY(dalloc(ctx, &ctx->Zw64, (size_t)ctx->N * ell * 8));
    TRY(dalloc(ctx, &ctx->U64, (size_t)ctx->ldP * ell * 8));
    CK(cudaMemsetAsync(ctx->U64, 0, (size_t)ctx->ldP * ell * 8, ctx->stream));
    TRY(dalloc(ctx, &ctx->Uh, (size_t)ctx->ldP * ((ell + 3) / 4 * 4) * 4));
    TRY(dalloc(ctx, &ctx->Ul, (size_t)ctx->ldP * ((ell + 3) / 4 * 4) * 4));
    TRY(dalloc(ctx, &ctx->w1p, (size_t)fused_pcg_blocks() * ell * sizeof(float2)));
    TRY(dalloc(ctx, &ctx->w2f, (size_t)ell * sizeof(float2)));
    CK(cudaMemsetAsync(ctx->Y64, 0, (size_t)ctx->ldP * ell * 8, ctx->stream));
    CK(cudaMemsetAsync(ctx->B64, 0, (size_t)ctx->ldP * ell * 8, ctx->stream));
  }
  ctx->ell_cap = ell;
  CK(cudaMemsetAsync(ctx->Om, 0, pe, ctx->stream));
  CK(cudaMemsetAsync(ctx->Y, 0, pe, ctx->stream));
  CK(cudaMemsetAsync(ctx->B, 0, pe, ctx->stream));
  CK(cudaMemsetAsync(ctx->U, 0, pe, ctx->stream));
  return NGD_OK;
}

ngd_status ensure_gpart(ngd_ctx* ctx, size_t elems) {
  if (elems <= ctx->gpart_elems) return NGD_OK;
  TRY(dalloc(ctx, &ctx->gpart, elems * 8));
  ctx->gpart_elems = elems;
  return NGD_OK;
}

// Number of K slices launch_gemm_df makes of K for a requested split count.
int split_count(int64_t K, int nsplit) {
  const int64_t kps = nsplit > 1 ? ((K + nsplit - 1) / nsplit + 15) / 16 * 16 : std::max<int64_t>(K, 1);
  return (int)((K + kps - 1) / kps);
}

// K-splits for an M x N output with a long K (tall-skinny products), so that ~1200 tiles run.
int choose_splits(int64_t M, int64_t N, int64_t K) {
  const int64_t tiles = ((M + 63) / 64) * ((N + 63) / 64);
  int64_t ns = std::max<int64_t>(1, 1200 / std::max<int64_t>(tiles, 1));
  ns = std::min<int64_t>(ns, std::max<int64_t>(1, K / 128));
  return (int)std::min<int64_t>(ns, 64);
}

// FP64 out = A^T B for column-major p x ell A and B (ld) -> ell x ell (column-major).
template <typename T>
ngd_status gram_atb(ngd_ctx* ctx, const T* A, const T* Bm, int64_t p, int64_t ld, int ell, double* out) {
  GemmArgs<T> g;
  g.M = ell; g.N = ell; g.K = p;
  g.A = A; g.sam = ld; g.sak = 1;
  g.B = Bm; g.sbk = 1; g.sbn = ld;
  g.nsplit = choose_splits(ell, ell, p);
  const int64_t kps = g.nsplit > 1 ? ((g.K + g.nsplit - 1) / g.nsplit + 15) / 16 * 16 : g.K;
  const int nz = (int)((g.K + kps - 1) / kps);
  TRY(ensure_gpart(ctx, (size_t)nz * ell * ell));
  g.out64 = ctx->gpart; g.split_stride = (int64_t)ell * ell;
  g.scm = 1; g.scn = ell;
  launch_gemm<T>(g, ctx->stream);
  launch_sum_splits(ctx->gpart, nz, (int64_t)ell * ell, (int64_t)ell * ell, out, ctx->stream);
  return check_launch(ctx);
}

// ------------------------------------------------------------------ linearization
template <typename T>
ngd_status prep_theta(ngd_ctx* ctx, const double* theta) {
  launch_prep_weights<T>(ctx->net, theta, (T*)ctx->prep, ctx->stream);
  ctx->tape_valid = false;
  ctx->prep_valid = true;
  return check_launch(ctx);
}

// Residuals, loss (scal[kSLoss]) and, in stored mode, the full Jacobian at theta.
template <typename T>
ngd_status linearize(ngd_ctx* ctx, const double* theta) {
  TRY(prep_theta<T>(ctx, theta));
  int nb;
  if (ctx->stored_j) {
    nb = launch_jacobian<T>(ctx->net, ctx->ps, (const T*)ctx->prep, 0, ctx->N, (T*)ctx->J, ctx->ldJ, ctx->r,
                            ctx->lpart, nullptr, 0, ctx->stream);
    if (nb <= 0) return set_err(ctx, NGD_ERR_UNSUPPORTED, "network too wide for the Jacobian kernel%s");
    // the fused matvec reads the weights as FP32 pairs (the caller owns w: re-split per linearization)
    if (ctx->whf) launch_split_df(ctx->ps.w, ctx->whf, ctx->whf + ctx->N, ctx->N, ctx->N, ctx->stream);
    ++ctx->j_version;
  } else {
    T* tape = ctx->tape_allowed ? (T*)ctx->tape : nullptr;
    nb = launch_forward<T>(ctx->net, ctx->ps, (const T*)ctx->prep, 0, ctx->N, ctx->r, ctx->lpart, tape, 0,
                           ctx->stream);
    if (nb <= 0) return set_err(ctx, NGD_ERR_UNSUPPORTED, "network too wide for the forward kernel%s");
    ctx->tape_valid = tape != nullptr;
  }
  launch_sum_partials(ctx->lpart, nb, 0.5, ctx->scal + kSLoss, ctx->stream);
  ctx->lin_valid = true;
  return check_launch(ctx);
}

// Workspace of the matrix-free VJP (allocated on first use).
template <typename T>
ngd_status ensure_rev(ngd_ctx* ctx) {
  if (ctx->rev_A) return NGD_OK;
  const NetDesc& net = ctx->net;
  const size_t per_row = ((size_t)3 * net.C * net.max_width + (size_t)net.tape_per_point + 1) * sizeof(T);
  ctx->rev_rows = std::max<int64_t>(32, std::min<int64_t>(ctx->N, (int64_t)((256ull << 20) / per_row)));
  const size_t buf = (size_t)ctx->rev_rows * net.C * net.max_width * sizeof(T);
  TRY(dalloc(ctx, &ctx->rev_A, buf));
  TRY(dalloc(ctx, &ctx->rev_X, buf));
  TRY(dalloc(ctx, &ctx->rev_Xb, buf));
  TRY(dalloc(ctx, &ctx->rev_tape, (size_t)ctx->rev_rows * net.tape_per_point * sizeof(T)));
  TRY(dalloc(ctx, &ctx->rev_ones, (size_t)ctx->rev_rows * sizeof(T)));
  std::vector<T> ones((size_t)ctx->rev_rows, T(1));
  CK(cudaMemcpy(ctx->rev_ones, ones.data(), ones.size() * sizeof(T), cudaMemcpyHostToDevice));
  return NGD_OK;
}

// K slices of a reduction GEMM with a tiles x K shape: enough blocks to fill the GPU, at least
// 256 terms per slice.  Returns the slice count launch_gemm will use.
template <typename T>
int rev_splits(GemmArgs<T>& g) {
  const int64_t tiles = ((g.M + 63) / 64) * ((g.N + 63) / 64);
  g.nsplit = (int)std::max<int64_t>(1, std::min<int64_t>((600 + tiles - 1) / tiles, g.K / 256));
  const int64_t kps = g.nsplit > 1 ? ((g.K + g.nsplit - 1) / g.nsplit + 15) / 16 * 16 : std::max<int64_t>(g.K, 1);
  return (int)std::max<int64_t>(1, (g.K + kps - 1) / kps);
}

// One layer product of the matrix-free J v / J^T c: FP32 contexts take the FP32 layer GEMM (K-slices
// of FP32 sums, FP64 slice partials), FP64 contexts the FP64 SIMT GEMM.  With g.out64 requested
// (reductions over points) the K-slice partials go to ctx->gpart and the slice count is returned;
// otherwise the product goes to g.outT in one slice.
template <typename T>
ngd_status layer_gemm(ngd_ctx* ctx, GemmArgs<T> g, bool reduce, int* nz_out) {
  int nz = 1;
  if (std::is_same<T, float>::value) {
    nz = reduce ? sgemm_layer_slices(g.M, g.N, g.K) : 1;
    if (reduce) {
      TRY(ensure_gpart(ctx, (size_t)nz * g.M * g.N));
      g.out64 = ctx->gpart;
      g.split_stride = g.M * g.N;
      g.outT = nullptr;
    }
    launch_sgemm_layer(reinterpret_cast<const GemmArgs<float>&>(g), nz, ctx->stream);
  } else {
    if (reduce) {
      nz = rev_splits(g);
      TRY(ensure_gpart(ctx, (size_t)nz * g.M * g.N));
      g.out64 = ctx->gpart;
      g.split_stride = g.M * g.N;
    }
    launch_gemm<T>(g, ctx->stream);
  }
  if (nz_out) *nz_out = nz;
  return NGD_OK;
}

// y = J^T c with J rows never formed: the reverse of the Taylor-mode forward by layers over chunks
// of points (Thm. 1; Sec. 4.1.2), the weight adjoint of each layer one GEMM over the chunk's
// points and channels, the input adjoint another.  The forward coefficients come from the stored
// tape when it is valid, else the chunk's forward is recomputed.
template <typename T>
ngd_status vjp_reverse(ngd_ctx* ctx, const double* cot, double* out) {
  TRY(ensure_rev<T>(ctx));
  const NetDesc& net = ctx->net;
  const int C = net.C, ldb = net.max_width, L = net.n_layers;
  const int64_t tpp = net.tape_per_point;
  int64_t toffs[kMaxLayers] = {};
  for (int l = 1; l < L - 1; ++l) toffs[l] = toffs[l - 1] + (int64_t)C * net.width[l];
  T* A = (T*)ctx->rev_A;
  T* X = (T*)ctx->rev_X;
  T* Xb = (T*)ctx->rev_Xb;
  const T* prep = (const T*)ctx->prep;
  for (int64_t r0 = 0; r0 < ctx->N; r0 += ctx->rev_rows) {
    const int64_t nr = std::min(ctx->rev_rows, ctx->N - r0);
    const T* tape = (const T*)ctx->tape;
    if (!ctx->tape_valid) {
      T* tb = (T*)ctx->rev_tape - r0 * tpp;        // the forward writes the tape of row r at tb + r * tpp
      if (launch_forward<T>(net, ctx->ps, prep, r0, nr, nullptr, nullptr, tb, 0, ctx->stream) <= 0)
        return set_err(ctx, NGD_ERR_UNSUPPORTED, "network too wide for the forward kernel%s");
      tape = tb;
    }
    launch_rev_seed<T>(net, ctx->ps, r0, nr, cot, A, ldb, ctx->stream);
    for (int l = L - 1; l >= 0; --l) {
      const int n_in = net.width[l], n_out = net.width[l + 1];
      const int64_t nW = (int64_t)n_out * n_in;
      launch_rev_input<T>(net, ctx->ps, l, tape, l >= 1 ? toffs[l - 1] : 0, r0, nr, X, ldb, ctx->stream);
      // W_bar_l = sum over (point, channel) rows of abar_l (outer) x_{l-1}
      GemmArgs<T> g;
      g.M = n_out; g.N = n_in; g.K = nr * C;
      g.A = A; g.sam = 1; g.sak = ldb;
      g.B = X; g.sbk = ldb; g.sbn = 1;
      g.scm = n_in; g.scn = 1;
      int nz = 1;
      TRY(layer_gemm<T>(ctx, g, true, &nz));
      launch_rev_sum(ctx->gpart, nz, nW, nW, out + net.theta_off[l], r0 > 0 ? 1 : 0, ctx->stream);
      // b_bar_l = sum over points of the value channel of abar_l
      GemmArgs<T> gb;
      gb.M = n_out; gb.N = 1; gb.K = nr;
      gb.A = A; gb.sam = 1; gb.sak = (int64_t)C * ldb;
      gb.B = (const T*)ctx->rev_ones; gb.sbk = 1; gb.sbn = 0;
      gb.scm = 1; gb.scn = 0;
      const int nzb = rev_splits(gb);
      TRY(ensure_gpart(ctx, (size_t)nzb * n_out));
      gb.out64 = ctx->gpart; gb.split_stride = n_out;
      launch_gemm<T>(gb, ctx->stream);
      launch_rev_sum(ctx->gpart, nzb, n_out, n_out, out + net.theta_off[l] + nW, r0 > 0 ? 1 : 0, ctx->stream);
      if (l == 0) break;
      // xbar_{l-1} = W_l^T abar_l for every (point, channel) row, then the adjoint through tanh
      GemmArgs<T> gx;
      gx.M = nr * C; gx.N = n_in; gx.K = n_out;
      gx.A = A; gx.sam = ldb; gx.sak = 1;
      gx.B = prep + net.wr_off[l]; gx.sbk = n_in; gx.sbn = 1;
      gx.outT = Xb; gx.scm = ldb; gx.scn = 1;
      TRY(layer_gemm<T>(ctx, gx, false, nullptr));
      launch_rev_tanh<T>(net, l - 1, tape, toffs[l - 1], r0, nr, Xb, A, ldb, ctx->stream);
    }
  }
  return check_launch(ctx);
}

// out = J v (FP64, N) for the tangent weights prept of v, by forward tangents by layers over chunks
// of points: per affine layer the pre-activation tangents of every (point, channel) row are
// X_{l-1} Wdot_l^T + Xdot_{l-1} W_l^T (two GEMMs), then the tangent through tanh (Thm. 1: the
// J v half of the Gramian matvec, the same layer arithmetic as vjp_reverse's).
template <typename T>
ngd_status jvp_layers(ngd_ctx* ctx, const T* prept, double* out) {
  TRY(ensure_rev<T>(ctx));
  const NetDesc& net = ctx->net;
  const int C = net.C, ldb = net.max_width, L = net.n_layers;
  const int64_t tpp = net.tape_per_point;
  int64_t toffs[kMaxLayers] = {};
  for (int l = 1; l < L - 1; ++l) toffs[l] = toffs[l - 1] + (int64_t)C * net.width[l];
  T* A = (T*)ctx->rev_A;
  T* X = (T*)ctx->rev_X;
  T* Xd = (T*)ctx->rev_Xb;
  const T* prep = (const T*)ctx->prep;
  for (int64_t r0 = 0; r0 < ctx->N; r0 += ctx->rev_rows) {
    const int64_t nr = std::min(ctx->rev_rows, ctx->N - r0);
    const T* tape = (const T*)ctx->tape;
    if (!ctx->tape_valid) {
      T* tb = (T*)ctx->rev_tape - r0 * tpp;
      if (launch_forward<T>(net, ctx->ps, prep, r0, nr, nullptr, nullptr, tb, 0, ctx->stream) <= 0)
        return set_err(ctx, NGD_ERR_UNSUPPORTED, "network too wide for the forward kernel%s");
      tape = tb;
    }
    for (int l = 0; l < L; ++l) {
      const int n_in = net.width[l], n_out = net.width[l + 1];
      launch_rev_input<T>(net, ctx->ps, l, tape, l >= 1 ? toffs[l - 1] : 0, r0, nr, X, ldb, ctx->stream);
      GemmArgs<T> g;
      g.M = nr * C; g.N = n_out; g.K = n_in;
      g.A = X; g.sam = ldb; g.sak = 1;
      g.B = prept + net.wr_off[l]; g.sbk = 1; g.sbn = n_in;
      g.outT = A; g.scm = ldb; g.scn = 1;
      TRY(layer_gemm<T>(ctx, g, false, nullptr));
      if (l >= 1) {
        GemmArgs<T> g2 = g;
        g2.A = Xd;
        g2.B = prep + net.wr_off[l];
        g2.accumulate = 1;
        TRY(layer_gemm<T>(ctx, g2, false, nullptr));
      }
      if (l < L - 1)
        launch_fwd_tangent<T>(net, l, tape, toffs[l], r0, nr, A, prept + net.b_off[l], Xd, ldb, ctx->stream);
      else
        launch_jvp_out<T>(net, ctx->ps, r0, nr, A, prept + net.b_off[l], ldb, out, ctx->stream);
    }
  }
  return check_launch(ctx);
}

// y = J^T c for the current prep: stored J (when valid), else the reverse pass by layers.
template <typename T>
ngd_status vjp_current(ngd_ctx* ctx, const double* cot, double* out, bool use_stored) {
  if (use_stored && ctx->stored_j && ctx->lin_valid) {
    if (std::is_same<T, float>::value)
      launch_coldot_df((const float*)ctx->J, ctx->ldJ, ctx->N, cot, ctx->colpart, ctx->colsplit, nullptr, ctx->stream);
    else
      launch_coldot<T>((const T*)ctx->J, ctx->ldJ, ctx->N, cot, ctx->colpart, ctx->colsplit, nullptr, ctx->stream);
    launch_coldot_finish(ctx->colpart, ctx->colsplit, ctx->p, ctx->ldJ, nullptr, 0.0, nullptr, out, 0, nullptr,
                         ctx->stream);
    return check_launch(ctx);
  }
  return vjp_reverse<T>(ctx, cot, out);
}

// y = (G + mu I) v at the current linearization.
template <typename T>
ngd_status gv_current(ngd_ctx* ctx, const double* v, double mu_h, const double* mu_d, double* y, const int* done) {
  if (ctx->stored_j) {
    if (std::is_same<T, float>::value && !done && ctx->yph) {
      // one pass over J in one cooperative kernel
      FusedPcgArgs fa;
      fa.J = (const float*)ctx->J; fa.ldJ = ctx->ldJ; fa.N = ctx->N; fa.p = ctx->p; fa.w = ctx->ps.w;
      fa.mu_d = mu_d; fa.mu_h = mu_h;
      fa.pv = const_cast<double*>(v); fa.q = y;
      fa.wh = ctx->whf; fa.wl = ctx->whf + ctx->N;
      fa.vhf = ctx->vhf; fa.vlf = ctx->vhf + ctx->ldJ;
      fa.yph = ctx->yph; fa.ypl = ctx->ypl; fa.red = ctx->fred;
      fa.mode = 1;
      const cudaError_t e = launch_pcg_fused(fa, ctx->stream);
      if (e != cudaErrorCooperativeLaunchTooLarge) {
        CK(e);
        return check_launch(ctx);
      }
      cudaGetLastError();
    }
    if (std::is_same<T, float>::value) {
      float* vh = (float*)ctx->vT;
      launch_split_df(v, vh, vh + ctx->ldJ, ctx->p, ctx->ldJ, ctx->stream);
      launch_rowdot_df((const float*)ctx->J, ctx->ldJ, ctx->N, vh, vh + ctx->ldJ, ctx->ps.w, nullptr, ctx->svec,
                       done, ctx->stream);
      launch_coldot_df((const float*)ctx->J, ctx->ldJ, ctx->N, ctx->svec, ctx->colpart, ctx->colsplit, done,
                       ctx->stream);
    } else {
      launch_d2t<T>(v, (T*)ctx->vT, ctx->p, ctx->ldJ, ctx->stream);
      launch_rowdot<T>((const T*)ctx->J, ctx->ldJ, ctx->N, (const T*)ctx->vT, ctx->ps.w, nullptr, ctx->svec, done,
                       ctx->stream);
      launch_coldot<T>((const T*)ctx->J, ctx->ldJ, ctx->N, ctx->svec, ctx->colpart, ctx->colsplit, done,
                       ctx->stream);
    }
    launch_coldot_finish(ctx->colpart, ctx->colsplit, ctx->p, ctx->ldJ, v, mu_h, mu_d, y, 0, done, ctx->stream);
    return check_launch(ctx);
  }
  // matrix-free: t = J v by forward tangents by layers, then y = J^T (w t) by the reverse by layers
  launch_prep_weights<T>(ctx->net, v, (T*)ctx->prep_t, ctx->stream);
  TRY(jvp_layers<T>(ctx, (const T*)ctx->prep_t, ctx->tvec));
  launch_mul(ctx->ps.w, ctx->tvec, ctx->svec, ctx->N, ctx->stream);
  TRY(vjp_current<T>(ctx, ctx->svec, y, false));
  launch_coldot_finish(nullptr, 0, ctx->p, ctx->p, v, mu_h, mu_d, y, 1, nullptr, ctx->stream);  // y += mu v
  return check_launch(ctx);
}

// ------------------------------------------------------------------ sketch and factor (internal buffers, ld = ldP)
// Explicit mantissa bits of the format the sketch Y is computed in: nu = eps(||Y||_F) in that
// format (the shift of App. A, read as MATLAB's eps of the sketch's precision).
int mantissa_bits(int prec) {
  switch (prec) {
    case NGD_SKETCH_DF: return 48;
    case NGD_SKETCH_TF32: return 10;
    case NGD_SKETCH_BF16: return 7;
    case NGD_SKETCH_F32: return 23;
    default: return 52;
  }
}

// FP64-accurate sketch (Y in float64): the tensor-core digit-plane form or the double-float form
bool acc64(int prec) { return prec == NGD_SKETCH_F64 || prec == NGD_SKETCH_DF; }

template <typename T>
ngd_status thin_qr_inplace(ngd_ctx* ctx, T* Om, int ell, bool tc) {
  // CholeskyQR: Om <- Om R^{-1}, R = chol(Om^T Om)^T (positive diagonal).  A Gaussian p x ell
  // matrix has condition number about (1 + sqrt(ell / p)) / (1 - sqrt(ell / p)) (<= 5/3 for
  // ell <= p / 16), so one pass leaves Q^T Q - I at a few units of the working precision; wider
  // test matrices take a second pass (CholeskyQR2).  With tc (FP32 Omega) the Gram matrix comes
  // FP64-accurate from the digit-plane tensor-core GEMM (its lower triangle, mirrored).
  const int passes = 16 * (int64_t)ell <= ctx->p ? 1 : 2;
  for (int pass = 0; pass < passes; ++pass) {
    bool done = false;
    if (tc && std::is_same<T, float>::value) {
      if (!ctx->oz) {
        ctx->oz = oz_create();
        if (!ctx->oz) return set_err(ctx, NGD_ERR_OOM, "tensor-core sketch state%s");
      }
      const char* why = nullptr;
      const cudaError_t e = oz_gram_self32(ctx->oz, (const float*)Om, ctx->p, ctx->ldP, ell, ctx->M, ell, &why,
                                           ctx->stream, ctx->status, ctx->wait_cycles);
      if (e == cudaErrorMemoryAllocation) return set_err(ctx, NGD_ERR_OOM, "tensor-core sketch workspace%s");
      CK(e);
      if (!why) {
        launch_mirror_lower(ctx->M, ell, ctx->stream);
        done = true;
      }
    }
    if (!done) {
      TRY(gram_atb<T>(ctx, Om, Om, ctx->p, ctx->ldP, ell, ctx->M));
      launch_symmetrize(ctx->M, ell, ctx->stream);
    }
    CK(launch_cholesky(ctx->M, ell, ctx->status, ctx->stream));
    launch_trsm_lt<T>(Om, ctx->ldP, ctx->p, ell, ctx->M, (T*)ctx->Lr, ctx->stream);
  }
  return check_launch(ctx);
}

ngd_status ensure_sampling(ngd_ctx* ctx) {
  if (ctx->gdiag) return NGD_OK;
  TRY(dalloc(ctx, &ctx->gdiag, (size_t)ctx->p * 8));
  TRY(dalloc(ctx, &ctx->samp_keys, (size_t)ctx->p * 8));
  TRY(dalloc(ctx, &ctx->samp_idx, (size_t)2048 * sizeof(int)));
  TRY(dalloc(ctx, &ctx->samp_count, sizeof(int)));
  // valid indices before the first selection: a failed selection leaves them in place
  CK(cudaMemsetAsync(ctx->samp_idx, 0, (size_t)2048 * sizeof(int), ctx->stream));
  return NGD_OK;
}

// diag(G) = sum_n w_n J[n, :]^2 (Eq. gram_diagonal) at the current linearization, into out (p):
// stored J read once; matrix-free J recomputed by point blocks.  FP64 partials over row slices,
// added in a fixed order.
template <typename T>
ngd_status gram_diag_internal(ngd_ctx* ctx, double* out) {
  const int64_t p = ctx->p;
  constexpr int kSplits = 64;
  TRY(ensure_gpart(ctx, (size_t)kSplits * p));
  int nz = 0;
  if (ctx->stored_j) {
    nz = launch_gram_diag<T>((const T*)ctx->J, ctx->ldJ, ctx->N, p, ctx->ps.w, ctx->gpart, p, kSplits, 0, ctx->stream);
  } else {
    for (int64_t r0 = 0; r0 < ctx->N; r0 += ctx->jrows) {
      const int64_t nr = std::min(ctx->jrows, ctx->N - r0);
      if (launch_jacobian<T>(ctx->net, ctx->ps, (const T*)ctx->prep, r0, nr, (T*)ctx->J, ctx->ldJ, nullptr, nullptr,
                             ctx->tape_valid ? (const T*)ctx->tape : nullptr, 0, ctx->stream) <= 0)
        return set_err(ctx, NGD_ERR_UNSUPPORTED, "network too wide for the Jacobian kernel%s");
      const int z = launch_gram_diag<T>((const T*)ctx->J, ctx->ldJ, nr, p, ctx->ps.w + r0, ctx->gpart, p, kSplits,
                                        r0 > 0 ? 1 : 0, ctx->stream);
      if (r0 == 0) nz = z;                 // the first block is the largest: it sets every partial
    }
  }
  launch_sum_splits(ctx->gpart, nz, p, p, out, ctx->stream);
  return check_launch(ctx);
}

// Y = J^T Zw for a stored J and Zw = diag(w) J Omega already formed (FP64-accurate form: Zw64, Y64)
ngd_status sketch_second_df(ngd_ctx* ctx, int ell) {
  GemmDfArgs<float, double> g2;
  g2.M = ctx->p; g2.N = ell; g2.K = ctx->N;
  g2.A = (const float*)ctx->J; g2.sam = 1; g2.sak = ctx->ldJ;
  g2.B = ctx->Zw64; g2.sbk = ell; g2.sbn = 1;
  g2.scm = 1; g2.scn = ctx->ldP;
  g2.nsplit = gemm_df_splits(g2.M, g2.N, g2.K);
  const int nz2 = split_count(g2.K, g2.nsplit);
  if (nz2 > 1) {
    TRY(ensure_gpart(ctx, (size_t)nz2 * ctx->ldP * ell));
    g2.out64 = ctx->gpart; g2.split_stride = (int64_t)ctx->ldP * ell;
    launch_gemm_df<float, double>(g2, ctx->stream);
    launch_sum_splits_t<double>(ctx->gpart, nz2, (int64_t)ctx->ldP * ell, ctx->p, ell, ctx->ldP, ctx->Y64, ctx->ldP,
                                ctx->stream);
  } else {
    g2.out64 = ctx->Y64;
    launch_gemm_df<float, double>(g2, ctx->stream);
  }
  return check_launch(ctx);
}

template <typename T>
ngd_status sketch_second_t(ngd_ctx* ctx, int ell) {
  GemmArgs<T> g2;
  g2.M = ctx->p; g2.N = ell; g2.K = ctx->N;
  g2.A = (const T*)ctx->J; g2.sam = 1; g2.sak = ctx->ldJ;
  g2.B = (const T*)ctx->Zw; g2.sbk = ell; g2.sbn = 1;
  g2.outT = (T*)ctx->Y; g2.scm = 1; g2.scn = ctx->ldP;
  launch_gemm<T>(g2, ctx->stream);
  return check_launch(ctx);
}

template <typename T>
ngd_status sketch_product(ngd_ctx* ctx, int ell, int prec);

// test_matrix: 0 Gaussian (Philox, thin QR); 1 columns of the identity sampled with probabilities
// proportional to diag G (the "sampling" test matrix of Sec. 3), already orthonormal.
template <typename T>
ngd_status sketch_internal(ngd_ctx* ctx, int ell, uint64_t seed, uint64_t step, int prec, int test_matrix = 0) {
  TRY(ensure_ell(ctx, ell));
  T* Om = (T*)ctx->Om;
  T* Y = (T*)ctx->Y;
  CK(cudaMemsetAsync(Om, 0, (size_t)ctx->ldP * ell * sizeof(T), ctx->stream));
  TRY(clear_status(ctx));
  if (test_matrix == 1) {
    TRY(ensure_sampling(ctx));
    TRY(gram_diag_internal<T>(ctx, ctx->gdiag));
    launch_sample_indices(ctx->gdiag, ctx->p, ell, seed, step, ctx->samp_keys, ctx->samp_idx, ctx->status,
                          ctx->stream);
    launch_selection_omega<T>(Om, ctx->ldP, ctx->samp_idx, ell, ctx->stream);
    // G Omega = G[:, S]: the first product is a gather of Jacobian columns
    if (ctx->stored_j && prec != NGD_SKETCH_TF32 && prec != NGD_SKETCH_BF16) {
      if (std::is_same<T, float>::value && acc64(prec)) {
        launch_gather_cols<float, double>((const float*)ctx->J, ctx->ldJ, ctx->N, ctx->samp_idx, ell, ctx->ps.w,
                                          ctx->Zw64, ctx->stream);
        return sketch_second_df(ctx, ell);
      }
      launch_gather_cols<T, T>((const T*)ctx->J, ctx->ldJ, ctx->N, ctx->samp_idx, ell, ctx->ps.w, (T*)ctx->Zw,
                               ctx->stream);
      return sketch_second_t<T>(ctx, ell);
    }
  } else {
    launch_philox_omega<T>(Om, ctx->ldP, ctx->p, ell, seed, step, ctx->stream);
    TRY(thin_qr_inplace<T>(ctx, Om, ell, prec == NGD_SKETCH_F64));
  }
  return sketch_product<T>(ctx, ell, prec);
}

// Y = G Omega for the Omega in ctx->Om (p x ell, ld ldP) in the arithmetic of prec: into ctx->Y64
// (FP64-accurate sketch of an F32 context) or ctx->Y.
template <typename T>
ngd_status sketch_product(ngd_ctx* ctx, int ell, int prec) {
  T* Om = (T*)ctx->Om;
  T* Y = (T*)ctx->Y;
  if (prec == NGD_SKETCH_TF32 || prec == NGD_SKETCH_BF16) {
    if (!std::is_same<T, float>::value) return set_err(ctx, NGD_ERR_INVALID_ARG, "TF32/BF16 sketch needs an F32 context%s");
    if (!ctx->stored_j) return set_err(ctx, NGD_ERR_UNSUPPORTED, "TF32/BF16 sketch needs the stored Jacobian%s");
    if (!ctx->tc) {
      ctx->tc = tc_create();
      if (!ctx->tc) return set_err(ctx, NGD_ERR_OOM, "tensor-core sketch state%s");
    }
    const char* why = nullptr;
    cudaError_t e = tc_sketch(ctx->tc, prec == NGD_SKETCH_BF16, (const float*)ctx->J, ctx->ldJ, ctx->N, ctx->p,
                              (const float*)Om, ctx->ldP, ell, ctx->ps.w, (float*)Y, &why, ctx->stream, ctx->status,
                              ctx->wait_cycles);
    if (why) return set_err(ctx, NGD_ERR_UNSUPPORTED, "tensor-core sketch: %s", why);
    CK(e);
    return check_launch(ctx);
  }
  if (std::is_same<T, float>::value && acc64(prec)) {
    if (!ctx->stored_j) return set_err(ctx, NGD_ERR_UNSUPPORTED, "the FP64-accurate sketch needs the stored Jacobian%s");
    if (prec == NGD_SKETCH_F64) {
      // FP64-accurate sketch on the tensor cores: exact sums of BF16 digit-plane products
      if (!ctx->oz) {
        ctx->oz = oz_create();
        if (!ctx->oz) return set_err(ctx, NGD_ERR_OOM, "tensor-core sketch state%s");
      }
      const char* why = nullptr;
      cudaError_t e = oz_sketch(ctx->oz, (const float*)ctx->J, ctx->ldJ, ctx->N, ctx->p, ctx->j_version, (const float*)Om,
                                ctx->ldP, ell, ctx->ps.w, ctx->Y64, &why, ctx->stream, ctx->status, ctx->wait_cycles);
      if (why) return set_err(ctx, NGD_ERR_UNSUPPORTED, "tensor-core sketch: %s", why);
      if (e == cudaErrorMemoryAllocation) return set_err(ctx, NGD_ERR_OOM, "tensor-core sketch workspace%s");
      CK(e);
      return check_launch(ctx);
    }
    // FP64-accurate sketch of the FP32 Jacobian (double-float arithmetic): Zw (FP64) = diag(w) J Om,
    // Y64 = J^T Zw.  The Nystrom core then resolves G's spectrum down to eps64 ||Y||, as in the paper.
    // K is split where that fills the GPU's block slots more evenly; the slices' FP64 partials
    // are then added in a fixed order
    GemmDfArgs<float, float> g1;
    g1.M = ctx->N; g1.N = ell; g1.K = ctx->p;
    g1.A = (const float*)ctx->J; g1.sam = ctx->ldJ; g1.sak = 1;
    g1.B = (const float*)Om; g1.sbk = 1; g1.sbn = ctx->ldP;
    g1.scm = ell; g1.scn = 1;
    g1.rowscale = ctx->ps.w;
    g1.nsplit = gemm_df_splits(g1.M, g1.N, g1.K);
    const int nz1 = split_count(g1.K, g1.nsplit);
    if (nz1 > 1) {
      TRY(ensure_gpart(ctx, (size_t)nz1 * ctx->N * ell));
      g1.out64 = ctx->gpart; g1.split_stride = (int64_t)ctx->N * ell;
      launch_gemm_df<float, float>(g1, ctx->stream);
      launch_sum_splits(ctx->gpart, nz1, (int64_t)ctx->N * ell, (int64_t)ctx->N * ell, ctx->Zw64, ctx->stream);
    } else {
      g1.out64 = ctx->Zw64;
      launch_gemm_df<float, float>(g1, ctx->stream);
    }
    GemmDfArgs<float, double> g2;
    g2.M = ctx->p; g2.N = ell; g2.K = ctx->N;
    g2.A = (const float*)ctx->J; g2.sam = 1; g2.sak = ctx->ldJ;
    g2.B = ctx->Zw64; g2.sbk = ell; g2.sbn = 1;
    g2.scm = 1; g2.scn = ctx->ldP;
    g2.nsplit = gemm_df_splits(g2.M, g2.N, g2.K);
    const int nz2 = split_count(g2.K, g2.nsplit);
    if (nz2 > 1) {
      TRY(ensure_gpart(ctx, (size_t)nz2 * ctx->ldP * ell));
      g2.out64 = ctx->gpart; g2.split_stride = (int64_t)ctx->ldP * ell;
      launch_gemm_df<float, double>(g2, ctx->stream);
      launch_sum_splits_t<double>(ctx->gpart, nz2, (int64_t)ctx->ldP * ell, ctx->p, ell, ctx->ldP, ctx->Y64, ctx->ldP,
                                  ctx->stream);
    } else {
      g2.out64 = ctx->Y64;
      launch_gemm_df<float, double>(g2, ctx->stream);
    }
    return check_launch(ctx);
  }
  if (ctx->stored_j) {
    // Zw = diag(w) J Om  (N x ell, row-major), then Y = J^T Zw  (p x ell, column-major)
    GemmArgs<T> g1;
    g1.M = ctx->N; g1.N = ell; g1.K = ctx->p;
    g1.A = (const T*)ctx->J; g1.sam = ctx->ldJ; g1.sak = 1;
    g1.B = Om; g1.sbk = 1; g1.sbn = ctx->ldP;
    g1.outT = (T*)ctx->Zw; g1.scm = ell; g1.scn = 1;
    g1.rowscale = ctx->ps.w;
    launch_gemm<T>(g1, ctx->stream);
    GemmArgs<T> g2;
    g2.M = ctx->p; g2.N = ell; g2.K = ctx->N;
    g2.A = (const T*)ctx->J; g2.sam = 1; g2.sak = ctx->ldJ;
    g2.B = (const T*)ctx->Zw; g2.sbk = ell; g2.sbn = 1;
    g2.outT = Y; g2.scm = 1; g2.scn = ctx->ldP;
    launch_gemm<T>(g2, ctx->stream);
    return check_launch(ctx);
  }
  // matrix-free: the same two products by point blocks whose Jacobian rows are recomputed
  // (Eq. G_matrixfree_batch), Y accumulated in FP64.
  const int64_t Bsz = ctx->jrows;
  TRY(ensure_gpart(ctx, (size_t)ctx->ldP * ell));
  for (int64_t r0 = 0; r0 < ctx->N; r0 += Bsz) {
    const int64_t nr = std::min(Bsz, ctx->N - r0);
    if (launch_jacobian<T>(ctx->net, ctx->ps, (const T*)ctx->prep, r0, nr, (T*)ctx->J, ctx->ldJ, nullptr, nullptr,
                           ctx->tape_valid ? (const T*)ctx->tape : nullptr, 0, ctx->stream) <= 0)
      return set_err(ctx, NGD_ERR_UNSUPPORTED, "network too wide for the Jacobian kernel%s");
    GemmArgs<T> g1;
    g1.M = nr; g1.N = ell; g1.K = ctx->p;
    g1.A = (const T*)ctx->J; g1.sam = ctx->ldJ; g1.sak = 1;
    g1.B = Om; g1.sbk = 1; g1.sbn = ctx->ldP;
    g1.outT = (T*)ctx->Zw; g1.scm = ell; g1.scn = 1;
    g1.rowscale = ctx->ps.w + r0;
    launch_gemm<T>(g1, ctx->stream);
    GemmArgs<T> g2;
    g2.M = ctx->p; g2.N = ell; g2.K = nr;
    g2.A = (const T*)ctx->J; g2.sam = 1; g2.sak = ctx->ldJ;
    g2.B = (const T*)ctx->Zw; g2.sbk = ell; g2.sbn = 1;
    g2.out64 = ctx->gpart; g2.split_stride = 0; g2.scm = 1; g2.scn = ctx->ldP;
    g2.accumulate = r0 > 0 ? 1 : 0;
    launch_gemm<T>(g2, ctx->stream);
  }
  launch_sum_splits_t<T>(ctx->gpart, 1, 0, ctx->p, ell, ctx->ldP, Y, ctx->ldP, ctx->stream);
  return check_launch(ctx);
}

// Factor of an FP64-accurate sketch in an FP32 context: Omega FP32 (exact values), Y, B and U in
// FP64.  The products Omega^T Y_nu, B^T B and U = B V Sigma^{-1} by the digit-plane tensor-core
// GEMM with the tensor-core sketch (prec NGD_SKETCH_F64), by the double-float GEMM otherwise.  U stays FP64: the apply of Alg. 4 scales the top
// directions by (lam_ell + mu) / (lam_1 + mu), ~1e-7 at later steps of the 5-D Poisson problem, a
// value formed by cancellation in I - U U^T that an FP32-rounded U perturbs by its own rounding.
// Lower triangle of C (ell x ell) = A^T B for the p x ell column-major operands (A = Omega in
// FP32, or A = B when Om is null) on the tensor cores; false when that path cannot serve.
bool oz_factor_gram(ngd_ctx* ctx, const float* Om, const double* B, int ell, double* C, ngd_status* st) {
  *st = NGD_OK;
  if (!ctx->oz) {
    ctx->oz = oz_create();
    if (!ctx->oz) {
      *st = set_err(ctx, NGD_ERR_OOM, "tensor-core sketch state%s");
      return true;
    }
  }
  const char* why = nullptr;
  const cudaError_t e = oz_gram_cols(ctx->oz, Om, B, ctx->p, ctx->ldP, ell, C, ell, &why, ctx->stream, ctx->status,
                                     ctx->wait_cycles);
  if (e == cudaErrorMemoryAllocation) {
    *st = set_err(ctx, NGD_ERR_OOM, "tensor-core factor workspace%s");
    return true;
  }
  if (e != cudaSuccess) {
    *st = set_err(ctx, NGD_ERR_CUDA, "CUDA: %s", cudaGetErrorString(e));
    return true;
  }
  return why == nullptr;
}

ngd_status factor_df(ngd_ctx* ctx, int ell, double shift_scale, int prec) {
  const float* Om = (const float*)ctx->Om;
  double* Bm = ctx->B64;
  const int64_t p = ctx->p, ld = ctx->ldP;
  TRY(clear_status(ctx));
  launch_frob2<double>(ctx->Y64, ld, p, ell, ctx->part, ctx->scal + kSFrob2, ctx->stream);
  // the double-float format carries 48 significant bits: nu = eps_48(||Y||_F)
  launch_compute_nu(ctx->scal + kSFrob2, 48, shift_scale, ctx->scal + kSNu, ctx->stream);
  launch_shift_add_mixed(ctx->Y64, Om, ctx->scal + kSNu, Bm, ld, p, ell, ctx->stream);      // Y_nu
  const bool tc = prec == NGD_SKETCH_F64;
  ngd_status st = NGD_OK;
  if (!(tc && oz_factor_gram(ctx, Om, Bm, ell, ctx->M, &st))) {
    GemmDfArgs<float, double> g;                                                           // Omega^T Y_nu
    g.M = ell; g.N = ell; g.K = p;
    g.A = Om; g.sam = ld; g.sak = 1;
    g.B = Bm; g.sbk = 1; g.sbn = ld;
    g.nsplit = gemm_df_splits(ell, ell, p, true);
    const int64_t kps = g.nsplit > 1 ? ((g.K + g.nsplit - 1) / g.nsplit + 15) / 16 * 16 : g.K;
    const int nz = (int)((g.K + kps - 1) / kps);
    TRY(ensure_gpart(ctx, (size_t)nz * ell * ell));
    g.out64 = ctx->gpart; g.split_stride = (int64_t)ell * ell; g.scm = 1; g.scn = ell;
    g.lower = 1;                                        // symmetric: the lower triangle, mirrored
    launch_gemm_df<float, double>(g, ctx->stream);
    launch_sum_splits(ctx->gpart, nz, (int64_t)ell * ell, (int64_t)ell * ell, ctx->M, ctx->stream);
  }
  TRY(st);
  launch_mirror_lower(ctx->M, ell, ctx->stream);
  CK(launch_cholesky(ctx->M, ell, ctx->status, ctx->stream));                                // = L L^T
  launch_trsm_lt<double>(Bm, ld, p, ell, ctx->M, (double*)ctx->eigws, ctx->stream);  // B = Y_nu L^{-T}
  if (!(tc && oz_factor_gram(ctx, nullptr, Bm, ell, ctx->V, &st))) {
    GemmDfArgs<double, double> g;                                                          // S = B^T B
    g.M = ell; g.N = ell; g.K = p;
    g.A = Bm; g.sam = ld; g.sak = 1;
    g.B = Bm; g.sbk = 1; g.sbn = ld;
    g.nsplit = gemm_df_splits(ell, ell, p, true);
    const int64_t kps = g.nsplit > 1 ? ((g.K + g.nsplit - 1) / g.nsplit + 15) / 16 * 16 : g.K;
    const int nz = (int)((g.K + kps - 1) / kps);
    TRY(ensure_gpart(ctx, (size_t)nz * ell * ell));
    g.out64 = ctx->gpart; g.split_stride = (int64_t)ell * ell; g.scm = 1; g.scn = ell;
    g.lower = 1;
    launch_gemm_df<double, double>(g, ctx->stream);
    launch_sum_splits(ctx->gpart, nz, (int64_t)ell * ell, (int64_t)ell * ell, ctx->V, ctx->stream);
  }
  TRY(st);
  launch_mirror_lower(ctx->V, ell, ctx->stream);
  CK(launch_sym_eig(ctx->V, ell, ctx->sig2, ctx->M, ctx->eigws, ctx->status, ctx->stream, ctx->dtype == NGD_F32));
  launch_nystrom_lambda(ctx->sig2, ctx->scal + kSNu, ell, ctx->lam, ctx->inv_sigma, ctx->stream);
  bool u_done = false;
  if (tc) {                                                                                // U = B V Sigma^{-1}
    const char* why = nullptr;
    const cudaError_t e = oz_gemm_bw(ctx->oz, Bm, ld, p, ell, ctx->M, ell, ctx->inv_sigma, ctx->U64, ld, &why,
                                     ctx->stream, ctx->status, ctx->wait_cycles);
    if (e == cudaErrorMemoryAllocation) return set_err(ctx, NGD_ERR_OOM, "tensor-core factor workspace%s");
    CK(e);
    u_done = why == nullptr;
  }
  if (!u_done) {
    GemmDfArgs<double, double> g;                                                          // U = B V Sigma^{-1}
    g.M = p; g.N = ell; g.K = ell;
    g.A = Bm; g.sam = 1; g.sak = ld;
    g.B = ctx->M; g.sbk = 1; g.sbn = ell;
    g.out64 = ctx->U64; g.scm = 1; g.scn = ld;
    g.colscale = ctx->inv_sigma;
    launch_gemm_df<double, double>(g, ctx->stream);
  }
  TRY(check_launch(ctx));
  return sync_status(ctx);
}

template <typename T>
ngd_status factor_internal(ngd_ctx* ctx, int ell, int prec, double shift_scale) {
  TRY(ensure_ell(ctx, ell));
  if (std::is_same<T, float>::value && acc64(prec)) return factor_df(ctx, ell, shift_scale, prec);
  const T* Om = (const T*)ctx->Om;
  const T* Y = (const T*)ctx->Y;
  T* Bm = (T*)ctx->B;
  TRY(clear_status(ctx));
  launch_frob2<T>(Y, ctx->ldP, ctx->p, ell, ctx->part, ctx->scal + kSFrob2, ctx->stream);
  launch_compute_nu(ctx->scal + kSFrob2, mantissa_bits(prec), shift_scale, ctx->scal + kSNu, ctx->stream);
  launch_shift_add<T>(Y, Om, ctx->scal + kSNu, Bm, ctx->ldP, ctx->p, ell, ctx->stream);   // Y_nu
  TRY(gram_atb<T>(ctx, Om, Bm, ctx->p, ctx->ldP, ell, ctx->M));                          // Omega^T Y_nu
  launch_symmetrize(ctx->M, ell, ctx->stream);
  CK(launch_cholesky(ctx->M, ell, ctx->status, ctx->stream));                            // = L L^T, C = L^T
  launch_trsm_lt<T>(Bm, ctx->ldP, ctx->p, ell, ctx->M, (T*)ctx->Lr, ctx->stream);  // B = Y_nu C^{-1}
  TRY(gram_atb<T>(ctx, Bm, Bm, ctx->p, ctx->ldP, ell, ctx->V));                          // S = B^T B
  launch_symmetrize(ctx->V, ell, ctx->stream);
  // S = V Sigma^2 V^T in FP64; sorted eigenvectors into M (free again after the triangular solve)
  CK(launch_sym_eig(ctx->V, ell, ctx->sig2, ctx->M, ctx->eigws, ctx->status, ctx->stream, ctx->dtype == NGD_F32));
  launch_nystrom_lambda(ctx->sig2, ctx->scal + kSNu, ell, ctx->lam, ctx->inv_sigma, ctx->stream);
  // U = B V_sorted diag(1/sigma)
  {
    const int64_t n2 = (int64_t)ell * ell;
    k_d2t_mat<T><<<(int)std::min<int64_t>((n2 + 255) / 256, 4096), 256, 0, ctx->stream>>>(ctx->M, ell, (T*)ctx->VsT,
                                                                                            ell, ell, ell); note_launch();
    GemmArgs<T> g;
    g.M = ctx->p; g.N = ell; g.K = ell;
    g.A = Bm; g.sam = 1; g.sak = ctx->ldP;
    g.B = (const T*)ctx->VsT; g.sbk = 1; g.sbn = ell;
    g.outT = (T*)ctx->U; g.scm = 1; g.scn = ctx->ldP;
    g.colscale = ctx->inv_sigma;
    launch_gemm<T>(g, ctx->stream);
  }
  TRY(check_launch(ctx));
  return sync_status(ctx);
}

// ------------------------------------------------------------------ PCG
ngd_status pcg_result(ngd_ctx* ctx, const PcgScalars* h, int* iters, double* relres) {
  if (iters) *iters = h->iters;
  if (relres) *relres = h->gn2 > 0 ? std::sqrt(h->rn2 / h->gn2) : 0.0;
  if (h->status & kStatBreakdown) return set_err(ctx, NGD_ERR_BREAKDOWN, "CG breakdown: p^T (G + mu I) p <= 0%s");
  if (h->status & kStatNonFinite) return set_err(ctx, NGD_ERR_NONFINITE, "non-finite value inside CG%s");
  return NGD_OK;
}

// P^{-1} v with U stored as float (u_f64 false) or double
void precond(ngd_ctx* ctx, bool u_f64, const void* U, int64_t ldU, int ell, const double* lam, double mu_h,
             const double* mu_d, const double* v, double* z, const int* done) {
  if (u_f64)
    launch_precond<double>((const double*)U, ldU, ctx->p, ell, lam, mu_h, mu_d, v, z, ctx->w1, done, ctx->stream);
  else
    launch_precond<float>((const float*)U, ldU, ctx->p, ell, lam, mu_h, mu_d, v, z, ctx->w1, done, ctx->stream);
}

// Arguments of the whole solve in one cooperative kernel for this context (FP32 stored J) on G
// blocks, with U split into its FP32 pair on the context stream; false when the context cannot
// take that kernel.  The solve's scalars (rtol, maxit) are already on the device.
template <typename T>
bool fused_args(ngd_ctx* ctx, const double* g, double mu_h, const double* mu_d, const void* U, bool u_f64,
                int64_t ldU, const double* lam, int ell, double* x, int G, FusedPcgArgs* out) {
  const bool pre = U != nullptr && ell > 0;
  const int64_t p = ctx->p;
  if (!std::is_same<T, float>::value || !ctx->stored_j || !ctx->yph ||
      !fused_pcg_supported_on(p, ctx->ldJ, pre ? ell : 0, G))
    return false;
  FusedPcgArgs fa;
  fa.J = (const float*)ctx->J; fa.ldJ = ctx->ldJ; fa.N = ctx->N; fa.p = p; fa.w = ctx->ps.w;
  if (pre) {
    if (u_f64)
      launch_split_transpose_df<double>((const double*)U, ldU, p, ell, ctx->Uh, ctx->Ul, ctx->stream);
    else
      launch_split_transpose_df<float>((const float*)U, ldU, p, ell, ctx->Uh, ctx->Ul, ctx->stream);
    fa.Uh = ctx->Uh; fa.Ul = ctx->Ul; fa.lam = lam; fa.ell = ell; fa.ldu = (ell + 3) / 4 * 4;
  }
  fa.mu_d = mu_d; fa.mu_h = mu_h;
  fa.g = g; fa.x = x; fa.r = ctx->rr; fa.z = ctx->z; fa.pv = ctx->pv; fa.q = ctx->q;
  fa.wh = ctx->whf; fa.wl = ctx->whf + ctx->N;
  fa.vhf = ctx->vhf; fa.vlf = ctx->vhf + ctx->ldJ;
  fa.yph = ctx->yph; fa.ypl = ctx->ypl; fa.red = ctx->fred; fa.w1p = ctx->w1p; fa.w2 = ctx->w2f;
  fa.sc = ctx->pcg; fa.mode = 0;
  fa.wait_cycles = ctx->wait_cycles;
  *out = fa;
  return true;
}

// The device scalars of a solve: rtol and maxit in, everything else cleared; the status word too.
ngd_status pcg_begin(ngd_ctx* ctx, double rtol, int maxit) {
  PcgScalars* h = ctx->h_pcg;
  memset(h, 0, sizeof(PcgScalars));
  h->rtol2 = rtol * rtol;
  h->maxit = maxit;
  CK(cudaMemcpyAsync(ctx->pcg, h, sizeof(PcgScalars), cudaMemcpyHostToDevice, ctx->stream));
  return clear_status(ctx);
}

template <typename T>
ngd_status pcg_internal(ngd_ctx* ctx, const double* g, double mu_h, const double* mu_d, const void* U, bool u_f64,
                        int64_t ldU, const double* lam, int ell, double rtol, int maxit, double* dout, int* iters,
                        double* relres) {
  PcgScalars* h = ctx->h_pcg;
  TRY(pcg_begin(ctx, rtol, maxit));
  const int64_t p = ctx->p;
  double* x = dout;
  double* r = ctx->rr;
  double* z = ctx->z;
  double* pv = ctx->pv;
  double* q = ctx->q;
  const bool pre = U != nullptr && ell > 0;
  const int* done = &ctx->pcg->done;
  FusedPcgArgs fa;
  if (fused_args<T>(ctx, g, mu_h, mu_d, U, u_f64, ldU, lam, ell, x, fused_pcg_blocks(), &fa)) {
    // the whole solve in one cooperative kernel (pcg_fused.cu)
    const cudaError_t e = launch_pcg_fused(fa, ctx->stream);
    if (e != cudaErrorCooperativeLaunchTooLarge) {
      CK(e);
      TRY(check_launch(ctx));
      CK(cudaMemcpyAsync(h, ctx->pcg, sizeof(PcgScalars), cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      return pcg_result(ctx, h, iters, relres);
    }
    cudaGetLastError();   // no co-resident grid: the multi-kernel solve below
  }
  launch_pcg_init(g, x, r, p, ctx->part, ctx->pcg, ctx->stream);
  if (pre) precond(ctx, u_f64, U, ldU, ell, lam, mu_h, mu_d, r, z, nullptr);
  launch_pcg_first_dir(r, pre ? z : r, pv, p, ctx->part, ctx->pcg, ctx->stream);
  TRY(check_launch(ctx));
  auto one_iteration = [&]() -> ngd_status {
    TRY(gv_current<T>(ctx, pv, mu_h, mu_d, q, done));
    launch_pcg_alpha(pv, q, p, ctx->part, ctx->pcg, ctx->stream);
    launch_pcg_update_xr(x, r, pv, q, p, ctx->part, ctx->pcg, ctx->stream);
    if (pre) precond(ctx, u_f64, U, ldU, ell, lam, mu_h, mu_d, r, z, done);
    launch_pcg_beta(r, pre ? z : r, p, ctx->part, ctx->pcg, ctx->stream);
    launch_pcg_update_p(pv, pre ? z : r, p, ctx->pcg, ctx->stream);
    return NGD_OK;
  };
  // The iterations are launch-bound at small sizes: `chunk` of them run as one CUDA graph, captured
  // once and replayed while U, lambda, mu, x and the linearization buffers stay the same.  The
  // kernels stop themselves on the device (done flag, maxit), so iterations past convergence in
  // the last replay return at once; the host reads the flag after each replay.  Matrix-free
  // matvecs do not check the flag, so that mode replays fewer iterations at a time.
  const int chunk = ctx->stored_j ? 8 : 2;
  const auto key_same = [&]() {
    const auto& k = ctx->pcg_key;
    return ctx->pcg_exec && k.U == U && k.u_f64 == u_f64 && k.ldU == ldU && k.lam == lam && k.ell == (pre ? ell : 0) &&
           k.mu_h == mu_h && k.mu_d == mu_d && k.x == x && k.chunk == chunk && k.J == ctx->J && k.prep == ctx->prep &&
           k.tape == ctx->tape_valid;
  };
  int launched = 0;
  bool converged = false;
  if (!key_same()) {
    if (ctx->pcg_exec) {
      cudaGraphExecDestroy(ctx->pcg_exec);
      ctx->pcg_exec = nullptr;
    }
    // one iteration for real first: it grows any workspace a matvec allocates on first use, which
    // a capture could not do
    TRY(one_iteration());
    ++launched;
    TRY(check_launch(ctx));
    CK(cudaMemcpyAsync(h, ctx->pcg, sizeof(PcgScalars), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    converged = h->done != 0;
    // the caller's stream may be the legacy default stream, which cannot be captured: capture on a
    // private stream (nothing runs during a capture) and replay on the caller's
    if (!ctx->cap_stream && cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
      ctx->cap_stream = nullptr;
    if (ctx->cap_stream) {
      cudaStream_t caller = ctx->stream;
      ctx->stream = ctx->cap_stream;
      const unsigned long long l0 = launches_now();
      cudaGraph_t graph = nullptr;
      ngd_status st = NGD_OK;
      if (cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        for (int k = 0; k < chunk && st == NGD_OK; ++k) st = one_iteration();
        const cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
        if (st == NGD_OK && e == cudaSuccess && graph &&
            cudaGraphInstantiate(&ctx->pcg_exec, graph, 0) == cudaSuccess) {
          ctx->pcg_key = {U, u_f64, ldU, lam, pre ? ell : 0, mu_h, mu_d, x, chunk, ctx->J, ctx->prep, ctx->tape_valid};
          ctx->pcg_graph_kernels = (int)(launches_now() - l0);
        } else {
          ctx->pcg_exec = nullptr;
        }
        if (graph) cudaGraphDestroy(graph);
      }
      ctx->stream = caller;
      g_launches.fetch_sub(launches_now() - l0, std::memory_order_relaxed);   // captured, not run
      cudaGetLastError();
    }
  }
  while (!converged && launched < maxit) {
    if (ctx->pcg_exec) {
      CK(cudaGraphLaunch(ctx->pcg_exec, ctx->stream));
      note_launch(ctx->pcg_graph_kernels);
      launched += chunk;
    } else {                                // no graph (capture refused): launch the iterations
      for (int k = 0; k < chunk && launched < maxit; ++k, ++launched) TRY(one_iteration());
    }
    TRY(check_launch(ctx));
    CK(cudaMemcpyAsync(h, ctx->pcg, sizeof(PcgScalars), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (h->done) break;
  }
  return pcg_result(ctx, h, iters, relres);
}

// lambda_1 of G at the current linearization by four steps of the power method (Alg. 2, Alg. 5):
// v0 the Gaussian column with counter word 2^32 - 2, v <- G v / ||G v||, the estimate the last
// Rayleigh quotient, into scal[kSLam1].  Uses z and q as scratch.
template <typename T>
ngd_status power_lambda1(ngd_ctx* ctx, uint64_t seed, uint64_t step) {
  const int64_t p = ctx->p;
  cudaStream_t st = ctx->stream;
  double* v = ctx->z;
  double* w = ctx->q;
  launch_philox_column(v, p, 0xFFFFFFFEu, seed, step, st);
  launch_dot(v, v, p, ctx->part, ctx->scal + kSDot, st);
  launch_scale_rsqrt(v, ctx->scal + kSDot, v, p, st);
  for (int it = 0; it < 4; ++it) {
    TRY(gv_current<T>(ctx, v, 0.0, nullptr, w, nullptr));
    launch_dot(v, w, p, ctx->part, ctx->scal + kSLam1, st);
    launch_dot(w, w, p, ctx->part, ctx->scal + kSDot, st);
    launch_scale_rsqrt(w, ctx->scal + kSDot, v, p, st);
  }
  return check_launch(ctx);
}

// Lower triangle of G = J^T diag(w) J (p x p, column-major, ldG) at the current linearization
// (stored J), FP64-accurate: for an FP32 Jacobian by the digit-plane tensor-core GEMM on the tiles
// of the lower triangle, otherwise w .* J in FP64 (ctx->Zfull) and the double-float GEMM on the
// lower triangle.
template <typename T>
ngd_status form_gramian(ngd_ctx* ctx, double* G, int64_t ldG) {
  const int64_t p = ctx->p;
  cudaStream_t st = ctx->stream;
  if (std::is_same<T, float>::value) {
    if (!ctx->oz) {
      ctx->oz = oz_create();
      if (!ctx->oz) return set_err(ctx, NGD_ERR_OOM, "tensor-core Gramian state%s");
    }
    const char* why = nullptr;
    const cudaError_t e = oz_gram(ctx->oz, (const float*)ctx->J, ctx->ldJ, ctx->N, p, ctx->ps.w, G, ldG, &why, st,
                                  ctx->status, ctx->wait_cycles);
    if (e == cudaErrorMemoryAllocation) return set_err(ctx, NGD_ERR_OOM, "tensor-core Gramian workspace%s");
    CK(e);
    if (!why) return check_launch(ctx);
  }
  if (!ctx->Zfull) TRY(dalloc(ctx, &ctx->Zfull, (size_t)ctx->N * ctx->ldJ * 8));
  launch_scale_rows_f64<T>((const T*)ctx->J, ctx->ldJ, ctx->N, ctx->ps.w, ctx->Zfull, st);
  GemmDfArgs<T, double> g;                                      // lower(G) = lower(J^T (w .* J))
  g.M = p; g.N = p; g.K = ctx->N;
  g.A = (const T*)ctx->J; g.sam = 1; g.sak = ctx->ldJ;
  g.B = ctx->Zfull; g.sbk = ctx->ldJ; g.sbn = 1;
  g.out64 = G; g.scm = 1; g.scn = ldG;
  g.lower = 1;
  launch_gemm_df<T, double>(g, st);
  return check_launch(ctx);
}

// NGD full (Alg. 2) direction at the current linearization (stored J) into ctx->d: lambda_1 by the
// power method, mu (into scal[kSMu]), G = J^T (w .* J) formed explicitly (FP64-accurate: for an
// FP32 Jacobian by the digit-plane tensor-core GEMM, otherwise w .* J in FP64 and the double-float
// GEMM on the lower triangle; mirrored from the lower one), G + mu I = L L^T (FP64 Cholesky:
// one cooperative kernel up to kCholBlockedMin - 1 unknowns, the blocked form above, its trailing
// updates on the digit-plane tensor-core GEMM for an FP32 Jacobian), d = L^{-T} L^{-1} g.
constexpr int64_t kCholBlockedMin = 768;
template <typename T>
ngd_status full_direction(ngd_ctx* ctx, const ngd_step_opts* o) {
  const int64_t p = ctx->p;
  const bool blocked = p >= kCholBlockedMin;
  cudaStream_t st = ctx->stream;
  if (!ctx->stored_j) return set_err(ctx, NGD_ERR_UNSUPPORTED, "NGD full needs the stored Jacobian%s");
  if (!ctx->Gfull) {
    ctx->ldG = blocked ? (p + 3) / 4 * 4 : p;                  // even: the blocked GEMMs stay vectorised
    TRY(dalloc(ctx, &ctx->Gfull, (size_t)ctx->ldG * p * 8));
    if (blocked) {
      TRY(dalloc(ctx, &ctx->chol_D, (size_t)256 * 256 * 8));
      TRY(dalloc(ctx, &ctx->chol_W, (size_t)256 * 256 * 8));
      TRY(dalloc(ctx, &ctx->chol_T, (size_t)256 * (p - 256) * 8));
    }
  }
  const int64_t ldG = ctx->ldG;
  TRY(clear_status(ctx));
  TRY(power_lambda1<T>(ctx, o->seed, o->step));
  launch_set_mu(ctx->scal + kSLam1, o->mu, o->gamma, ctx->scal + kSLoss, o->mu_loss_coef, ctx->scal + kSMu, st);
  TRY(form_gramian<T>(ctx, ctx->Gfull, ldG));
  launch_lower_to_upper(ctx->Gfull, p, ldG, st);
  launch_copy_diag(ctx->Gfull, p, ldG, ctx->x, st);          // x: scratch for diag(G)
  launch_add_diag_dev(ctx->Gfull, p, ldG, ctx->scal + kSMu, st);
  // A mu below the rounding of the formed G (mu = 10 eps lambda_1 late in training) can leave
  // G + mu I numerically indefinite; the paper is silent on failures, and the factorization is
  // retried with 8 mu, 64 mu, ..., 8^5 mu (both Cholesky forms write only the lower triangle: it
  // is rebuilt from the upper one and the saved diagonal).
  for (int attempt = 0;; ++attempt) {
    if (blocked)
      CK(launch_cholesky_blocked(ctx->Gfull, p, ldG, ctx->status, ctx->chol_D, ctx->chol_W, ctx->chol_T, st,
                                 std::is_same<T, float>::value ? ctx->oz : nullptr, ctx->wait_cycles));
    else
      CK(launch_cholesky(ctx->Gfull, (int)p, ctx->status, st));
    CK(cudaMemcpyAsync(ctx->h_int, ctx->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (!(ctx->h_int[0] & kStatNotSpd) || (ctx->h_int[0] & kStatTimeout)) break;
    if (attempt + 1 >= kShiftAttempts)
      return set_err(ctx, NGD_ERR_NOT_SPD, "NGD full: G + mu I is not positive definite up to 8^5 mu%s");
    TRY(clear_status(ctx));
    launch_scale_scalar(ctx->scal + kSMu, 8.0, st);
    launch_restore_lower(ctx->Gfull, p, ldG, ctx->x, ctx->scal + kSMu, st);
  }
  TRY(sync_status(ctx));
  CK(launch_chol_solve(ctx->Gfull, (int)p, ldG, ctx->g, ctx->d, ctx->z, st));
  return check_launch(ctx);
}

// RPCholNGD preconditioner (Alg. 5) at the current linearization (stored J): diag G, lambda_1 by
// four power-method steps (start: the Gaussian column with word 2^32 - 2), mu (into scal[kSMu]),
// block RPCholesky (rounds of o->rpchol_block pivots, at most o->ell columns, stopping when the
// residual trace is below mu p), then the thin SVD F = U Sigma V^T by eig(F^T F) in FP64, so that
// P^{-1} = U (Sigma^2 + mu I)^{-1} U^T + mu^{-1} (I - U U^T) (Eq. rpchol_svdprecond), which equals
// the Woodbury form (Eq. rpchol_precond).  It is handed to pCG as a Nystrom-form preconditioner
// with lambda = Sigma^2 and one appended zero column and eigenvalue, whose scaled form mu times
// the above: *ell_pc = rank + 1 (0 when no column was found: P = mu I).  Outputs: U (FP64, ld ldP)
// in *Uout, rank, lambda_1.
template <typename T>
ngd_status rpchol_build(ngd_ctx* ctx, const ngd_step_opts* o, int* ell_pc, int* rank, double* lam1_out,
                        const double** Uout) {
  const int64_t p = ctx->p, ld = ctx->ldP;
  const int b = o->rpchol_block, t = o->ell / o->rpchol_block;
  const bool f32 = std::is_same<T, float>::value;
  if (!ctx->stored_j) return set_err(ctx, NGD_ERR_UNSUPPORTED, "RPCholNGD needs the stored Jacobian%s");
  TRY(ensure_ell(ctx, o->ell + 1));
  TRY(ensure_sampling(ctx));
  TRY(ensure_gpart(ctx, (size_t)o->ell * b));
  double* F = f32 ? ctx->B64 : (double*)ctx->B;         // p x ell
  double* Cb = f32 ? ctx->Y64 : (double*)ctx->Y;        // p x b residual block
  double* Zb = f32 ? ctx->Zw64 : (double*)ctx->Zw;      // N x b: diag(w) J[:, S']
  double* Uo = f32 ? ctx->U64 : (double*)ctx->U;
  cudaStream_t st = ctx->stream;
  TRY(clear_status(ctx));
  TRY(gram_diag_internal<T>(ctx, ctx->gdiag));
  TRY(power_lambda1<T>(ctx, o->seed, o->step));
  launch_set_mu(ctx->scal + kSLam1, o->mu, o->gamma, ctx->scal + kSLoss, o->mu_loss_coef, ctx->scal + kSMu, st);
  CK(cudaMemcpyAsync(ctx->h_scal, ctx->scal, kSCount * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const double mu = ctx->h_scal[kSMu];
  *lam1_out = ctx->h_scal[kSLam1];
  if (!(mu > 0.0) || !std::isfinite(mu)) return set_err(ctx, NGD_ERR_NONFINITE, "RPCholNGD: mu is not positive%s");
  const double eps = mu * (double)p;
  double trace = 0.0;
  {
    std::vector<double> dh((size_t)p);
    CK(cudaMemcpyAsync(dh.data(), ctx->gdiag, (size_t)p * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (double x : dh) trace += x > 0.0 ? x : 0.0;
  }
  int r = 0;
  for (int i = 0; i < t && trace >= eps; ++i) {
    launch_rpchol_pivots(ctx->gdiag, p, b, i, o->seed, o->step, ctx->perm, ctx->samp_idx, ctx->samp_count, st);
    CK(cudaMemcpyAsync(ctx->h_int, ctx->samp_count, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const int nsel = ctx->h_int[0];
    if (nsel <= 0) break;
    // C = G[:, S'] - F F[S', :]^T
    if (f32) {
      launch_gather_cols<float, double>((const float*)ctx->J, ctx->ldJ, ctx->N, ctx->samp_idx, nsel, ctx->ps.w, Zb, st);
      GemmDfArgs<float, double> g;
      g.M = p; g.N = nsel; g.K = ctx->N;
      g.A = (const float*)ctx->J; g.sam = 1; g.sak = ctx->ldJ;
      g.B = Zb; g.sbk = nsel; g.sbn = 1;
      g.out64 = Cb; g.scm = 1; g.scn = ld;
      launch_gemm_df<float, double>(g, st);
    } else {
      launch_gather_cols<double, double>((const double*)ctx->J, ctx->ldJ, ctx->N, ctx->samp_idx, nsel, ctx->ps.w, Zb,
                                         st);
      GemmArgs<double> g;
      g.M = p; g.N = nsel; g.K = ctx->N;
      g.A = (const double*)ctx->J; g.sam = 1; g.sak = ctx->ldJ;
      g.B = Zb; g.sbk = nsel; g.sbn = 1;
      g.outT = Cb; g.scm = 1; g.scn = ld;
      launch_gemm<double>(g, st);
    }
    if (r > 0) {
      launch_gather_rows_neg(F, ld, ctx->samp_idx, nsel, r, ctx->gpart, st);
      GemmDfArgs<double, double> g;
      g.M = p; g.N = nsel; g.K = r;
      g.A = F; g.sam = 1; g.sak = ld;
      g.B = ctx->gpart; g.sbk = 1; g.sbn = r;
      g.out64 = Cb; g.scm = 1; g.scn = ld;
      g.accumulate = 1;
      launch_gemm_df<double, double>(g, st);
    }
    // R = chol(C[S', S']); new columns C R^{-1}; a pivot block that is not positive definite ends
    // the factorization with the columns found so far
    launch_pivot_block(Cb, ld, ctx->samp_idx, nsel, ctx->M, st);
    CK(launch_cholesky(ctx->M, nsel, ctx->status, st));
    CK(cudaMemcpyAsync(ctx->h_int, ctx->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (ctx->h_int[0] & kStatTimeout) return sync_status(ctx);
    if (ctx->h_int[0] & kStatNotSpd) {
      CK(cudaMemsetAsync(ctx->status, 0, sizeof(int), st));
      break;
    }
    double* Fn = F + (int64_t)r * ld;
    CK(cudaMemcpy2DAsync(Fn, (size_t)ld * 8, Cb, (size_t)ld * 8, (size_t)p * 8, nsel, cudaMemcpyDeviceToDevice, st));
    launch_trsm_lt<double>(Fn, ld, p, nsel, ctx->M, ctx->A1, st);
    const int nb = launch_rpchol_diag(ctx->gdiag, Fn, ld, p, nsel, ctx->samp_idx, ctx->part, st);
    launch_sum_partials(ctx->part, nb, 1.0, ctx->scal + kSTrace, st);
    CK(cudaMemcpyAsync(ctx->h_scal + kSTrace, ctx->scal + kSTrace, 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    trace = ctx->h_scal[kSTrace];
    r += nsel;
  }
  *rank = r;
  *Uout = Uo;
  if (r == 0) {
    *ell_pc = 0;
    return check_launch(ctx);
  }
  // thin SVD of F by eig(F^T F)
  {
    GemmDfArgs<double, double> g;
    g.M = r; g.N = r; g.K = p;
    g.A = F; g.sam = ld; g.sak = 1;
    g.B = F; g.sbk = 1; g.sbn = ld;
    g.nsplit = choose_splits(r, r, p);
    const int nz = split_count(g.K, g.nsplit);
    TRY(ensure_gpart(ctx, (size_t)nz * r * r));
    g.out64 = ctx->gpart; g.split_stride = (int64_t)r * r; g.scm = 1; g.scn = r;
    launch_gemm_df<double, double>(g, st);
    launch_sum_splits(ctx->gpart, nz, (int64_t)r * r, (int64_t)r * r, ctx->V, st);
  }
  launch_symmetrize(ctx->V, r, st);
  CK(launch_sym_eig(ctx->V, r, ctx->sig2, ctx->M, ctx->eigws, ctx->status, st, ctx->dtype == NGD_F32));
  launch_rpchol_lambda(ctx->sig2, r, ctx->lam, ctx->inv_sigma, st);
  {
    GemmDfArgs<double, double> g;                                                      // U = F V Sigma^{-1}
    g.M = p; g.N = r; g.K = r;
    g.A = F; g.sam = 1; g.sak = ld;
    g.B = ctx->M; g.sbk = 1; g.sbn = r;
    g.out64 = Uo; g.scm = 1; g.scn = ld;
    g.colscale = ctx->inv_sigma;
    launch_gemm_df<double, double>(g, st);
  }
  CK(cudaMemsetAsync(Uo + (int64_t)r * ld, 0, (size_t)ld * 8, st));                  // the appended column
  *ell_pc = r + 1;
  TRY(check_launch(ctx));
  return sync_status(ctx);
}

template <typename T>
ngd_status loss_at(ngd_ctx* ctx, const double* theta, double* loss_host) {
  TRY(prep_theta<T>(ctx, theta));
  const int nb = launch_forward<T>(ctx->net, ctx->ps, (const T*)ctx->prep, 0, ctx->N, nullptr, ctx->lpart, nullptr, 0,
                                   ctx->stream);
  if (nb <= 0) return set_err(ctx, NGD_ERR_UNSUPPORTED, "network too wide for the forward kernel%s");
  launch_sum_partials(ctx->lpart, nb, 0.5, ctx->scal + kSLoss, ctx->stream);
  CK(cudaMemcpyAsync(ctx->h_scal + kSLoss, ctx->scal + kSLoss, 8, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  *loss_host = ctx->h_scal[kSLoss];
  ctx->lin_valid = false;
  ctx->prep_valid = false;
  return check_launch(ctx);
}

float ev_ms(ngd_ctx* ctx, int a, int b) {
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ctx->ev[a], ctx->ev[b]);
  return ms;
}

// NVTX ranges around the phases of a step (host-side annotations for profilers; no-ops otherwise).
// The range stack stays balanced on every return path.
struct PhaseRange {
  bool open = false;
  void next(const char* name) {
    if (open) nvtxRangePop();
    nvtxRangePushA(name);
    open = true;
  }
  ~PhaseRange() {
    if (open) nvtxRangePop();
  }
};

// State of one NGD step between its stages (a batch runs the stages of many problems in turn).
struct StepState {
  ngd_step_info inf{};
  bool rpchol = false, full = false;
  int ell_pc = 0, rp_rank = 0;
  double rp_lam1 = 0.0;
  bool u_f64 = true;
  const void* Ust = nullptr;
  int iters = 0;
  double relres = 0.0;
};

// Stage 1 of a step: gradient and linearization, then the preconditioner (Nystrom sketch and
// factor with the damping, RPCholesky) or NGD full's direction.
template <typename T>
ngd_status step_prepare(ngd_ctx* ctx, double* theta, const ngd_step_opts* o, StepState& st) {
  ngd_step_info& inf = st.inf;
  inf = ngd_step_info{};
  PhaseRange phase;
  phase.next("linearize");
  CK(cudaEventRecord(ctx->ev[0], ctx->stream));
  // Alg. 1, gradient: at theta (and the linearization the matvecs use)
  TRY(linearize<T>(ctx, theta));
  launch_mul(ctx->ps.w, ctx->r, ctx->svec, ctx->N, ctx->stream);
  TRY(vjp_current<T>(ctx, ctx->svec, ctx->g, true));
  CK(cudaEventRecord(ctx->ev[1], ctx->stream));
  const bool rpchol = st.rpchol = o->precond == NGD_PRECOND_RPCHOL;
  const bool full = st.full = o->precond == NGD_DIRECT_FULL;
  int& ell_pc = st.ell_pc;
  ell_pc = o->ell;
  st.rp_rank = 0;
  st.rp_lam1 = 0.0;
  bool& u_f64 = st.u_f64;
  u_f64 = true;
  const void*& Ust = st.Ust;               // taken after the factor: the workspace grows on demand
  Ust = nullptr;
  if (rpchol) {
    // Alg. 5: RPCholesky preconditioner (its mu comes from the power-method lambda_1)
    phase.next("rpchol");
    CK(cudaEventRecord(ctx->ev[2], ctx->stream));
    const double* Urp = nullptr;
    TRY(rpchol_build<T>(ctx, o, &ell_pc, &st.rp_rank, &st.rp_lam1, &Urp));
    Ust = Urp;
    u_f64 = true;
    CK(cudaEventRecord(ctx->ev[3], ctx->stream));
  } else if (full) {
    // Alg. 2: the direction by Cholesky of the explicit G + mu I (no pCG)
    phase.next("full");
    CK(cudaEventRecord(ctx->ev[2], ctx->stream));
    TRY(full_direction<T>(ctx, o));
    ell_pc = 0;
    CK(cudaEventRecord(ctx->ev[3], ctx->stream));
  } else {
    phase.next("sketch");
    // Alg. 4, randomized Nystrom (App. A): fresh Omega from (seed, step)
    TRY(sketch_internal<T>(ctx, o->ell, o->seed, o->step, o->sketch, o->test_matrix));
    CK(cudaEventRecord(ctx->ev[2], ctx->stream));
    phase.next("factor");
    double scale = 1.0;
    ngd_status fs = NGD_OK;
    for (int attempt = 0; attempt < kShiftAttempts; ++attempt) {
      fs = factor_internal<T>(ctx, o->ell, o->sketch, scale);
      if (fs != NGD_ERR_NOT_SPD) break;
      inf.shift_retries++;
      scale *= 8.0;
    }
    if (fs != NGD_OK) return fs;
    CK(cudaEventRecord(ctx->ev[3], ctx->stream));
    // Alg. 4, damping: mu fixed, gamma eps lambda_1, or the Sec. 5 maximum with c L^2
    launch_set_mu(ctx->lam, o->mu, o->gamma, ctx->scal + kSLoss, o->mu_loss_coef, ctx->scal + kSMu, ctx->stream);
    u_f64 = !std::is_same<T, float>::value || acc64(o->sketch);
    Ust = std::is_same<T, float>::value && acc64(o->sketch) ? (const void*)ctx->U64 : ctx->U;
  }
  return NGD_OK;
}

// Stage 2: the direction by pCG on (G + mu I) d = g with the preconditioner of Alg. 4 or Alg. 5
// (Alg. 3); nothing for NGD full.
template <typename T>
ngd_status step_solve(ngd_ctx* ctx, const ngd_step_opts* o, StepState& st) {
  PhaseRange phase;
  phase.next("pcg");
  st.iters = 0;
  st.relres = 0.0;
  if (!st.full)
    TRY(pcg_internal<T>(ctx, ctx->g, 0.0, ctx->scal + kSMu, st.Ust, st.u_f64, ctx->ldP, ctx->lam, st.ell_pc, o->rtol,
                        o->maxit, ctx->d, &st.iters, &st.relres));
  CK(cudaEventRecord(ctx->ev[4], ctx->stream));
  return NGD_OK;
}

// Stage 3: Armijo line search along theta - alpha d, the update, the next rank and the step's info.
template <typename T>
ngd_status step_finish(ngd_ctx* ctx, double* theta, const ngd_step_opts* o, StepState& st, ngd_step_info* info) {
  ngd_step_info& inf = st.inf;
  const int64_t p = ctx->p;
  const bool rpchol = st.rpchol, full = st.full;
  const int ell_pc = st.ell_pc, rp_rank = st.rp_rank;
  const double rp_lam1 = st.rp_lam1;
  const int iters = st.iters;
  const double relres = st.relres;
  PhaseRange phase;
  phase.next("linesearch");
  // Alg. 1, line search: Armijo backtracking along theta - alpha d
  launch_dot(ctx->g, ctx->d, p, ctx->part, ctx->scal + kSDot, ctx->stream);
  CK(cudaMemcpyAsync(ctx->h_scal, ctx->scal, kSCount * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  const double L0 = ctx->h_scal[kSLoss], slope = ctx->h_scal[kSDot], mu = ctx->h_scal[kSMu];
  const double nu = (rpchol || full) ? 0.0 : ctx->h_scal[kSNu];
  std::vector<double> lam_all((size_t)std::max(ell_pc, 1), 0.0);
  if (ell_pc > 0) {
    CK(cudaMemcpyAsync(lam_all.data(), ctx->lam, (size_t)ell_pc * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
  }
  double lam_h[2] = {lam_all[0], lam_all[(size_t)std::max(ell_pc, 1) - 1]};
  int ell_next = o->ell;
  if (rpchol) {
    // lambda_1 from the power method; the smallest kept sigma^2 of F; the rank RPCholesky found
    lam_h[0] = rp_lam1;
    lam_h[1] = 0.0;
    for (int i = 0; i + 1 < ell_pc; ++i)
      if (lam_all[(size_t)i] > 0.0) lam_h[1] = lam_all[(size_t)i];
    ell_next = rp_rank;
  } else if (full) {
    lam_h[0] = ctx->h_scal[kSLam1];          // the power-method estimate
    lam_h[1] = 0.0;
  } else if (o->ell_max > 0) {
    // Alg. 4: rank of the next step's sketch
    if (lam_h[1] > 10.0 * mu) {
      ell_next = std::min(o->ell + o->ell_delta, o->ell_max);
    } else {
      int first = -1;                      // first 0-based index with lambda_hat < 10 mu
      for (int i = 0; i < o->ell; ++i)
        if (lam_all[(size_t)i] < 10.0 * mu) {
          first = i;
          break;
        }
      ell_next = first < 0 ? o->ell : std::min(first + 2, o->ell_max);
    }
  }
  double alpha = 1.0, L1 = L0;
  int trials = 0;
  bool accepted = false;
  for (; trials < o->armijo_max;) {
    ++trials;
    launch_axpy_to(theta, ctx->d, alpha, ctx->theta_trial, p, ctx->stream);
    double Lt = 0.0;
    TRY(loss_at<T>(ctx, ctx->theta_trial, &Lt));
    if (std::isfinite(Lt) && Lt <= L0 - o->armijo_c1 * alpha * slope) {
      L1 = Lt;
      accepted = true;
      break;
    }
    alpha *= o->armijo_rho;
  }
  if (!accepted) alpha = 0.0;
  // Alg. 1, update
  if (alpha != 0.0) launch_axpy_to(theta, ctx->d, alpha, theta, p, ctx->stream);
  CK(cudaEventRecord(ctx->ev[5], ctx->stream));
  CK(cudaEventSynchronize(ctx->ev[5]));
  ctx->lin_valid = false;
  ctx->tape_valid = false;
  ctx->prep_valid = false;
  inf.loss_before = L0;
  inf.loss_after = L1;
  inf.alpha = alpha;
  inf.mu = mu;
  inf.nu = nu;
  inf.lam1 = lam_h[0];
  inf.lam_ell = lam_h[1];
  inf.relres = relres;
  inf.pcg_iters = iters;
  inf.armijo_trials = trials;
  inf.status = 0;
  inf.ms_linearize = ev_ms(ctx, 0, 1);
  inf.ms_sketch = ev_ms(ctx, 1, 2);
  inf.ms_factor = ev_ms(ctx, 2, 3);
  inf.ms_pcg = ev_ms(ctx, 3, 4);
  inf.ms_linesearch = ev_ms(ctx, 4, 5);
  inf.ell_next = ell_next;
  if (info) *info = inf;
  return check_launch(ctx);
}

template <typename T>
ngd_status step_impl(ngd_ctx* ctx, double* theta, const ngd_step_opts* o, ngd_step_info* info) {
  StepState st;
  TRY(step_prepare<T>(ctx, theta, o, st));
  TRY(step_solve<T>(ctx, o, st));
  return step_finish<T>(ctx, theta, o, st, info);
}

}  // namespace

static bool valid_prec(int prec) { return prec >= NGD_SKETCH_F64 && prec <= NGD_SKETCH_DF; }

// Host checks of ngd_step's options against the context.
static ngd_status check_step_opts(ngd_ctx* ctx, const ngd_step_opts* o) {
  if (o->ell < 1 || o->ell > std::min<int64_t>(ctx->p, 2048) || !(o->rtol >= 0.0) || o->maxit < 1 ||
      !valid_prec(o->sketch) || !(o->armijo_rho > 0.0 && o->armijo_rho < 1.0) || o->armijo_max < 1 ||
      !(o->mu_loss_coef >= 0.0) || o->ell_max < 0 || o->ell_max > std::min<int64_t>(ctx->p, 2048) ||
      o->ell_delta < 0 || o->test_matrix < 0 || o->test_matrix > 1 || o->precond < 0 || o->precond > 2 ||
      (o->precond == NGD_PRECOND_RPCHOL && (o->rpchol_block < 1 || o->rpchol_block > o->ell || o->ell > 2047)))
    return set_err(ctx, NGD_ERR_INVALID_ARG, "bad step options%s");
  if (ctx->dtype == NGD_F64 && o->sketch != NGD_SKETCH_F64)
    return set_err(ctx, NGD_ERR_INVALID_ARG, "an F64 context sketches in F64 only%s");
  return NGD_OK;
}

// ====================================================================== C ABI
extern "C" {

void ngd_default_step_opts(ngd_step_opts* o) {
  if (!o) return;
  o->ell = 100;
  o->mu = 0.0;
  o->gamma = 10.0;
  o->rtol = 1e-6;
  o->maxit = 500;
  o->sketch = NGD_SKETCH_F64;
  o->seed = 0;
  o->step = 0;
  o->armijo_c1 = 1e-4;
  o->armijo_rho = 0.5;
  o->armijo_max = 30;
  o->mu_loss_coef = 0.0;
  o->ell_max = 0;
  o->ell_delta = 20;
  o->test_matrix = 0;
  o->precond = 0;
  o->rpchol_block = 20;
}

ngd_status ngd_create(const ngd_problem_desc* desc, ngd_ctx** out) {
  ngd_ctx* ctx = nullptr;
  if (!out) return NGD_ERR_INVALID_ARG;
  *out = nullptr;
  if (!desc || !desc->widths || !desc->X || !desc->w || !desc->target) return NGD_ERR_INVALID_ARG;
  const int L = desc->n_layers;
  if (L < 2 || L > kMaxLayers) return NGD_ERR_INVALID_ARG;
  const int d = desc->widths[0];
  if (d < 1 || d > kMaxD || desc->widths[L] != 1) return NGD_ERR_INVALID_ARG;
  for (int l = 1; l < L; ++l)
    if (desc->widths[l] < 1 || desc->widths[l] > kMaxWidth) return NGD_ERR_INVALID_ARG;
  if (desc->n_int < 0 || desc->n_bnd < 0 || desc->n_int + desc->n_bnd < 1) return NGD_ERR_INVALID_ARG;
  if (desc->pde != NGD_PDE_POISSON && desc->pde != NGD_PDE_HEAT) return NGD_ERR_INVALID_ARG;
  if (desc->pde == NGD_PDE_HEAT && d < 2) return NGD_ERR_INVALID_ARG;
  if (desc->dtype != NGD_F64 && desc->dtype != NGD_F32) return NGD_ERR_INVALID_ARG;
  if (desc->gv_mode < NGD_GV_AUTO || desc->gv_mode > NGD_GV_MATRIX_FREE) return NGD_ERR_INVALID_ARG;

  ctx = new (std::nothrow) ngd_ctx();
  if (!ctx) return NGD_ERR_OOM;
  NetDesc& net = ctx->net;
  net.n_layers = L;
  net.d = d;
  net.C = d + 2;
  net.pde = desc->pde;
  net.kappa = desc->kappa;
  int64_t off = 0, wsum = 0, bsum = 0, hsum = 0;
  int maxw = 1;
  for (int l = 0; l <= L; ++l) net.width[l] = desc->widths[l];
  for (int l = 0; l < L; ++l) {
    const int64_t ni = net.width[l], no = net.width[l + 1];
    net.theta_off[l] = off;
    off += no * ni + no;
    wsum += no * ni;
    bsum += no;
    if (l >= 1) maxw = std::max(maxw, (int)ni);
    if (l < L - 1) hsum += no;
  }
  net.max_width = maxw;
  net.p = off;
  int64_t o1 = 0;
  for (int l = 0; l < L; ++l) {
    net.wt_off[l] = o1;
    o1 += (int64_t)net.width[l + 1] * net.width[l];
  }
  for (int l = 0; l < L; ++l) {
    net.wr_off[l] = o1;
    o1 += (int64_t)net.width[l + 1] * net.width[l];
  }
  for (int l = 0; l < L; ++l) {
    net.b_off[l] = o1;
    o1 += net.width[l + 1];
  }
  net.prep_size = o1;
  net.tape_per_point = (int64_t)net.C * hsum;
  (void)wsum; (void)bsum;

  ctx->ps.X = desc->X;
  ctx->ps.w = desc->w;
  ctx->ps.target = desc->target;
  ctx->ps.n_int = desc->n_int;
  ctx->ps.N = desc->n_int + desc->n_bnd;
  ctx->dtype = desc->dtype;
  ctx->gv_mode = desc->gv_mode;
  ctx->mem_budget = desc->mem_budget;
  ctx->stream = (cudaStream_t)desc->stream;
  ctx->elt = desc->dtype == NGD_F32 ? 4 : 8;
  ctx->N = ctx->ps.N;
  ctx->p = net.p;
  ctx->ldJ = round_up(net.p, 32);
  ctx->ldP = round_up(net.p, 32);

  auto fail = [&](ngd_status st) {
    ngd_destroy(ctx);
    return st;
  };
  // the Taylor kernels stage whole points in shared memory: at least one tile of 4 (C <= 8 channels)
  // or 2 points for the Jacobian, 2 or 1 for the JVP, must fit the 200 KB budget
  const size_t jac_pts = net.C <= 8 ? 4 : 2, jvp_pts = net.C <= 8 ? 2 : 1;
  if (jac_smem_per_point(net, ctx->elt) * jac_pts > 200 * 1024 ||
      jvp_smem_per_point(net, ctx->elt) * jvp_pts > 200 * 1024)
    return fail(NGD_ERR_UNSUPPORTED);

  const size_t jbytes = (size_t)ctx->N * ctx->ldJ * ctx->elt;
  if (ctx->gv_mode == NGD_GV_STORED_J)
    ctx->stored_j = true;
  else if (ctx->gv_mode == NGD_GV_MATRIX_FREE)
    ctx->stored_j = false;
  else
    ctx->stored_j = ctx->mem_budget == 0 || jbytes <= ctx->mem_budget;
  const size_t tbytes = (size_t)ctx->N * net.tape_per_point * ctx->elt;
  const size_t used = ctx->stored_j ? jbytes : 0;
  ctx->tape_allowed = ctx->mem_budget == 0 ? !ctx->stored_j : (used + tbytes <= ctx->mem_budget);

  if (ctx->stored_j) {
    ctx->jrows = ctx->N;
  } else {
    const int64_t rows = (int64_t)((64ull << 20) / ((size_t)ctx->ldJ * ctx->elt));
    ctx->jrows = std::max<int64_t>(32, std::min<int64_t>(rows, ctx->N));
  }
  const int vn = ctx->elt == 4 ? 4 : 2;
  ctx->colsplit = coldot_nsplit(ctx->N, ctx->ldJ, vn);
  const int64_t N = ctx->N, p = ctx->p;
  if (dalloc(ctx, &ctx->J, (size_t)ctx->jrows * ctx->ldJ * ctx->elt) != NGD_OK) return fail(NGD_ERR_OOM);
  if (ctx->tape_allowed && dalloc(ctx, &ctx->tape, tbytes) != NGD_OK) return fail(NGD_ERR_OOM);
  if (dalloc(ctx, &ctx->prep, net.prep_size * ctx->elt) != NGD_OK || dalloc(ctx, &ctx->prep_t, net.prep_size * ctx->elt) != NGD_OK ||
      dalloc(ctx, &ctx->vT, 2 * ctx->ldJ * ctx->elt) != NGD_OK || dalloc(ctx, &ctx->r, N * 8) != NGD_OK ||
      dalloc(ctx, &ctx->svec, N * 8) != NGD_OK || dalloc(ctx, &ctx->tvec, N * 8) != NGD_OK ||
      dalloc(ctx, &ctx->lpart, N * 8) != NGD_OK || dalloc(ctx, &ctx->part, kRedBlocks * 8) != NGD_OK ||
      dalloc(ctx, &ctx->colpart, (size_t)ctx->colsplit * ctx->ldJ * 8) != NGD_OK ||
      dalloc(ctx, &ctx->scal, kSCount * 8) != NGD_OK || dalloc(ctx, &ctx->status, 16) != NGD_OK ||
      dalloc(ctx, &ctx->pcg, sizeof(PcgScalars)) != NGD_OK || dalloc(ctx, &ctx->x, p * 8) != NGD_OK ||
      dalloc(ctx, &ctx->rr, p * 8) != NGD_OK || dalloc(ctx, &ctx->z, p * 8) != NGD_OK ||
      dalloc(ctx, &ctx->pv, p * 8) != NGD_OK || dalloc(ctx, &ctx->q, p * 8) != NGD_OK ||
      dalloc(ctx, &ctx->g, p * 8) != NGD_OK || dalloc(ctx, &ctx->d, p * 8) != NGD_OK ||
      dalloc(ctx, &ctx->theta_trial, p * 8) != NGD_OK)
    return fail(NGD_ERR_OOM);
  if (ctx->dtype == NGD_F32 && ctx->stored_j && fused_pcg_supported(p, ctx->ldJ, 0)) {
    const size_t nb = (size_t)fused_pcg_blocks();
    if (dalloc(ctx, &ctx->yph, nb * ctx->ldJ * 4) != NGD_OK || dalloc(ctx, &ctx->ypl, nb * ctx->ldJ * 4) != NGD_OK ||
        dalloc(ctx, &ctx->fred, nb * 4 * 8) != NGD_OK || dalloc(ctx, &ctx->vhf, 2 * ctx->ldJ * 4) != NGD_OK ||
        dalloc(ctx, &ctx->whf, 2 * N * 4) != NGD_OK)
      return fail(NGD_ERR_OOM);
    if (cudaMemsetAsync(ctx->vhf, 0, 2 * ctx->ldJ * 4, ctx->stream) != cudaSuccess) return fail(NGD_ERR_CUDA);
  }
  if (cudaMallocHost((void**)&ctx->h_scal, kSCount * 8) != cudaSuccess ||
      cudaMallocHost((void**)&ctx->h_int, 16 * sizeof(int)) != cudaSuccess ||
      cudaMallocHost((void**)&ctx->h_pcg, sizeof(PcgScalars)) != cudaSuccess)
    return fail(NGD_ERR_OOM);
  for (auto& e : ctx->ev)
    if (cudaEventCreate(&e) != cudaSuccess) return fail(NGD_ERR_CUDA);
  if (cudaMemsetAsync(ctx->J, 0, (size_t)ctx->jrows * ctx->ldJ * ctx->elt, ctx->stream) != cudaSuccess ||
      cudaMemsetAsync(ctx->status, 0, 16, ctx->stream) != cudaSuccess ||
      cudaMemsetAsync(ctx->scal, 0, kSCount * 8, ctx->stream) != cudaSuccess)
    return fail(NGD_ERR_CUDA);
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return fail(NGD_ERR_CUDA);
  *out = ctx;
  return NGD_OK;
}

void ngd_destroy(ngd_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  void* dev[] = {ctx->prep, ctx->prep_t, ctx->J, ctx->tape, ctx->vT, ctx->r, ctx->svec, ctx->tvec, ctx->part,
                 ctx->lpart, ctx->colpart, ctx->scal, ctx->status, ctx->pcg, ctx->x, ctx->rr, ctx->z, ctx->pv, ctx->q,
                 ctx->g, ctx->d, ctx->theta_trial, ctx->Om, ctx->Y, ctx->B, ctx->U, ctx->Lr, ctx->VsT, ctx->Zw, ctx->M,
                 ctx->A1, ctx->V, ctx->Vs, ctx->sig2, ctx->inv_sigma, ctx->lam, ctx->dinv, ctx->w1, ctx->gpart,
                 ctx->perm, ctx->eigws, ctx->Y64, ctx->B64, ctx->Zw64, ctx->U64, ctx->Uh, ctx->Ul,
                 ctx->yph, ctx->ypl, ctx->fred, ctx->w1p, ctx->w2f, ctx->vhf, ctx->whf, ctx->gdiag,
                 ctx->samp_keys, ctx->samp_idx, ctx->samp_count, ctx->Gfull, ctx->Zfull, ctx->chol_D,
                 ctx->chol_W, ctx->chol_T, ctx->rev_A, ctx->rev_X, ctx->rev_Xb, ctx->rev_tape, ctx->rev_ones};
  for (void* pp : dev)
    if (pp) cudaFree(pp);
  if (ctx->h_scal) cudaFreeHost(ctx->h_scal);
  if (ctx->h_int) cudaFreeHost(ctx->h_int);
  if (ctx->h_pcg) cudaFreeHost(ctx->h_pcg);
  for (auto& e : ctx->ev)
    if (e) cudaEventDestroy(e);
  if (ctx->tc) tc_destroy(ctx->tc);
  if (ctx->oz) oz_destroy(ctx->oz);
  if (ctx->pcg_exec) cudaGraphExecDestroy(ctx->pcg_exec);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  delete ctx;
}

uint64_t ngd_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

const char* ngd_last_error(const ngd_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }
int64_t ngd_num_params(const ngd_ctx* ctx) { return ctx ? ctx->p : -1; }
int64_t ngd_num_points(const ngd_ctx* ctx) { return ctx ? ctx->N : -1; }

ngd_status ngd_set_wait_limit(ngd_ctx* ctx, int64_t cycles) {
  if (!ctx) return NGD_ERR_INVALID_ARG;
  if (cycles < 1) return set_err(ctx, NGD_ERR_INVALID_ARG, "the wait limit must be >= 1 cycle%s");
  ctx->wait_cycles = (long long)cycles;
  return NGD_OK;
}

ngd_status ngd_set_stream(ngd_ctx* ctx, void* stream) {
  if (!ctx) return NGD_ERR_INVALID_ARG;
  ctx->stream = (cudaStream_t)stream;
  return NGD_OK;
}

ngd_status ngd_residual(ngd_ctx* ctx, const double* theta, double* r, double* loss) {
  if (!ctx) return NGD_ERR_INVALID_ARG;
  if (!theta) return set_err(ctx, NGD_ERR_INVALID_ARG, "theta is NULL%s");
  return by_dtype(ctx, [&](auto z) -> ngd_status {
    using T = decltype(z);
    TRY(prep_theta<T>(ctx, theta));
    T* tape = ctx->tape_allowed ? (T*)ctx->tape : nullptr;
    const int nb = launch_forward<T>(ctx->net, ctx->ps, (const T*)ctx->prep, 0, ctx->N, r ? r : ctx->r, ctx->lpart,
                                     tape, 0, ctx->stream);
    if (nb <= 0) return set_err(ctx, NGD_ERR_UNSUPPORTED, "network too wide for the forward kernel%s");
    launch_sum_partials(ctx->lpart, nb, 0.5, ctx->scal + kSLoss, ctx->stream);
    ctx->tape_valid = tape != nullptr;
    ctx->lin_valid = !ctx->stored_j;
    TRY(check_launch(ctx));
    if (loss) {
      CK(cudaMemcpyAsync(ctx->h_scal + kSLoss, ctx->scal + kSLoss, 8, cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      *loss = ctx->h_scal[kSLoss];
    }
    return NGD_OK;
  });
}

ngd_status ngd_eval(ngd_ctx* ctx, const double* theta, double* out) {
  if (!ctx) return NGD_ERR_INVALID_ARG;
  if (!theta || !out) return set_err(ctx, NGD_ERR_INVALID_ARG, "theta/out is NULL%s");
  return by_dtype(ctx, [&](auto z) -> ngd_status {
    using T = decltype(z);
    TRY(prep_theta<T>(ctx, theta));
    const int nb = launch_forward<T>(ctx->net, ctx->ps, (const T*)ctx->prep, 0, ctx->N, ctx->r, ctx->lpart, nullptr,
                                     0, ctx->stream, out);
    if (nb <= 0) return set_err(ctx, NGD_ERR_UNSUPPORTED, "network too wide for the forward kernel%s");
    launch_sum_partials(ctx->lpart, nb, 0.5, ctx->scal + kSLoss, ctx->stream);
    ctx->tape_valid = false;
    ctx->lin_valid = !ctx->stored_j;
    return check_launch(ctx);
  });
}

ngd_status ngd_jvp(ngd_ctx* ctx, const double* theta, const double* v, double* out) {
  if (!ctx) return NGD_ERR_INVALID_ARG;
  if (!v || !out) return set_err(ctx, NGD_ERR_INVALID_ARG, "v/out is NULL%s");
  if (!theta && !ctx->prep_valid && !(ctx->stored_j && ctx->lin_valid))
    return set_err(ctx, NGD_ERR_INVALID_ARG, "theta is NULL and the context holds no parameters%s");
  return by_dtype(ctx, [&](auto z) -> ngd_status {
    using T = decltype(z);
    if (theta) {
      TRY(prep_theta<T>(ctx, theta));
      ctx->lin_valid = !ctx->stored_j;
    }
    launch_prep_weights<T>(ctx->net, v, (T*)ctx->prep_t, ctx->stream);
    if (launch_jvp<T>(ctx->net, ctx->ps, (const T*)ctx->prep, (const T*)ctx->prep_t, out, 0, ctx->stream) <= 0)
      return set_err(ctx, NGD_ERR_UNSUPPORTED, "network too wide for the JVP kernel%s");
    return check_launch(ctx);
  });
}

ngd_status ngd_vjp(ngd_ctx* ctx, const double* theta, const double* cot, double* out) {
  if (!ctx) return NGD_ERR_INVALID_ARG;
  if (!cot || !out) return set_err(ctx, NGD_ERR_INVALID_ARG, "cot/out is NULL%s");
  if (!theta && !ctx->prep_valid && !(ctx->stored_j && ctx->lin_valid))
    return set_err(ctx, NGD_ERR_INVALID_ARG, "theta is NULL and the context holds no parameters%s");
  return by_dtype(ctx, [&](auto z) -> ngd_status {
    using T = decltype(z);
    if (theta) {
      TRY(prep_theta<T>(ctx, theta));
      ctx->lin_valid = !ctx->stored_j;
    }
    // stored J serves only when nothing newer (theta, tape) was prepared since it was formed
    return vjp_current<T>(ctx, cot, out, theta == nullptr && !ctx->tape_valid);
  });
}

ngd_status ngd_gradient(ngd_ctx* ctx, const double* theta, double* g, double* r, double* loss) {
  if (!ctx) return NGD_ERR_INVALID_ARG;
  if (!theta || !g) return set_err(ctx, NGD_ERR_INVALID_ARG, "theta/g is NULL%s");
  return by_dtype(ctx, [&](auto z) -> ngd_status {
    using T = decltype(z);
    TRY(linearize<T>(ctx, theta));
    launch_mul(ctx->ps.w, ctx->r, ctx->svec, ctx->N, ctx->stream);
    TRY(vjp_current<T>(ctx, ctx->svec, g, true));
    if (r) CK(cudaMemcpyAsync(r, ctx->r, ctx->N * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    if (loss) {
      CK(cudaMemcpyAsync(ctx->h_scal + kSLoss, ctx->scal + kSLoss, 8, cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      *loss = ctx->h_scal[kSLoss];
    }
    return check_launch(ctx);
  });
}

ngd_status ngd_set_jacobian(ngd_ctx* ctx, const void* J, int64_t ldJ) {
  if (!ctx) return NGD_ERR_INVALID_ARG;
  if (!J || ldJ < ctx->p) return set_err(ctx, NGD_ERR_INVALID_ARG, "J is NULL or ldJ < p%s");
  if (!ctx->stored_j) return set_err(ctx, NGD_ERR_UNSUPPORTED, "the context does not store its Jacobian%s");
  const size_t row = (size_t)ctx->p * ctx->elt;
  // the padding columns p .. ldJ-1 of the context's J stay zero (set at creation, never written)
  CK(cudaMemcpy2DAsync(ctx->J, (size_t)ctx->ldJ * ctx->elt, J, (size_t)ldJ * ctx->elt, row, (size_t)ctx->N,
                       cudaMemcpyDeviceToDevice, ctx->stream));
  if (ctx->whf) launch_split_df(ctx->ps.w, ctx->whf, ctx->whf + ctx->N, ctx->N, ctx->N, ctx->stream);
  ctx->tape_valid = false;
  ctx->lin_valid = true;
  ++ctx->j_version;
  return check_launch(ctx);
}

ngd_status ngd_gramian_mv(ngd_ctx* ctx, const double* theta, const double* v, double mu, double* y) {
  if (!ctx) return NGD_ERR_INVALID_ARG;
  if (!v || !y || v == y) return set_err(ctx, NGD_ERR_INVALID_ARG, "v/y NULL or aliased%s");
  if (!(mu >= 0.0)) return set_err(ctx, NGD_ERR_INVALID_ARG, "mu must be >= 0%s");
  return by_dtype(ctx, [&](auto z) -> ngd_status {
    using T = decltype(z);
    if (theta) TRY(linearize<T>(ctx, theta));
    if (!ctx->lin_valid) return set_err(ctx, NGD_ERR_INVALID_ARG, "no linearization: pass theta%s");
    return gv_current<T>(ctx, v, mu, nullptr, y, nullptr);
  });
}


ngd_status ngd_nystrom_sketch(ngd_ctx* ctx, const double* theta, int ell, uint64_t seed, uint64_t step, int prec,
                              void* Omega, void* Y) {
  if (!ctx) return NGD_ERR_INVALID_ARG;
  if (!Omega || !Y) return set_err(ctx, NGD_ERR_INVALID_ARG, "Omega/Y is NULL%s");
  if (ell < 1 || ell > std::min<int64_t>(ctx->p, 2048)) return set_err(ctx, NGD_ERR_INVALID_ARG, "ell out of range%s");
  if (!valid_prec(prec)) return set_err(ctx, NGD_ERR_INVALID_ARG, "bad sketch precision%s");
  if (ctx->dtype == NGD_F64 && prec != NGD_SKETCH_F64)
    return set_err(ctx, NGD_ERR_INVALID_ARG, "an F64 context sketches in F64 only%s");
  return by_dtype(ctx, [&](auto z) -> ngd_status {
    using T = decltype(z);
    if (theta) TRY(linearize<T>(ctx, theta));
    if (!ctx->lin_valid) return set_err(ctx, NGD_ERR_INVALID_ARG, "no linearization: pass theta%s");
    TRY(sketch_internal<T>(ctx, ell, seed, step, prec));
    TRY(sync_status(ctx));
    const size_t w = (size_t)ctx->p * sizeof(T), sp = (size_t)ctx->ldP * sizeof(T);
    CK(cudaMemcpy2DAsync(Omega, w, ctx->Om, sp, w, ell, cudaMemcpyDeviceToDevice, ctx->stream));
    if (std::is_same<T, float>::value && acc64(prec))
      CK(cudaMemcpy2DAsync(Y, (size_t)ctx->p * 8, ctx->Y64, (size_t)ctx->ldP * 8, (size_t)ctx->p * 8, ell,
                           cudaMemcpyDeviceToDevice, ctx->stream));
    else
      CK(cudaMemcpy2DAsync(Y, w, ctx->Y, sp, w, ell, cudaMemcpyDeviceToDevice, ctx->stream));
    return check_launch(ctx);
  });
}

ngd_status ngd_gramian_mm(ngd_ctx* ctx, const double* theta, int ell, const void* V, int64_t ldV, int prec, void* Y,
                          int64_t ldY) {
  if (!ctx) return NGD_ERR_INVALID_ARG;
  if (!V || !Y || V == Y) return set_err(ctx, NGD_ERR_INVALID_ARG, "V/Y NULL or aliased%s");
  if (ell < 1 || ell > std::min<int64_t>(ctx->p, 2048) || ldV < ctx->p || ldY < ctx->p)
    return set_err(ctx, NGD_ERR_INVALID_ARG, "ell out of range or ldV/ldY < p%s");
  if (!valid_prec(prec)) return set_err(ctx, NGD_ERR_INVALID_ARG, "bad sketch precision%s");
  if (ctx->dtype == NGD_F64 && prec != NGD_SKETCH_F64)
    return set_err(ctx, NGD_ERR_INVALID_ARG, "an F64 context sketches in F64 only%s");
  return by_dtype(ctx, [&](auto z) -> ngd_status {
    using T = decltype(z);
    if (theta) TRY(linearize<T>(ctx, theta));
    if (!ctx->lin_valid) return set_err(ctx, NGD_ERR_INVALID_ARG, "no linearization: pass theta%s");
    TRY(ensure_ell(ctx, ell));
    const size_t w = (size_t)ctx->p * sizeof(T), sp = (size_t)ctx->ldP * sizeof(T);
    // rows p .. ldP-1 of the internal copy stay zero: the products read whole padded columns
    CK(cudaMemsetAsync(ctx->Om, 0, sp * ell, ctx->stream));
    CK(cudaMemcpy2DAsync(ctx->Om, sp, V, (size_t)ldV * sizeof(T), w, ell, cudaMemcpyDeviceToDevice, ctx->stream));
    TRY(clear_status(ctx));
    TRY(sketch_product<T>(ctx, ell, prec));
    TRY(sync_status(ctx));
    if (std::is_same<T, float>::value && acc64(prec))
      CK(cudaMemcpy2DAsync(Y, (size_t)ldY * 8, ctx->Y64, (size_t)ctx->ldP * 8, (size_t)ctx->p * 8, ell,
                           cudaMemcpyDeviceToDevice, ctx->stream));
    else
      CK(cudaMemcpy2DAsync(Y, (size_t)ldY * sizeof(T), ctx->Y, sp, w, ell, cudaMemcpyDeviceToDevice, ctx->stream));
    return check_launch(ctx);
  });
}

ngd_status ngd_gramian_full(ngd_ctx* ctx, const double* theta, double* G, int64_t ldG) {
  if (!ctx) return NGD_ERR_INVALID_ARG;
  if (!G || ldG < ctx->p) return set_err(ctx, NGD_ERR_INVALID_ARG, "G is NULL or ldG < p%s");
  if (!ctx->stored_j) return set_err(ctx, NGD_ERR_UNSUPPORTED, "the explicit Gramian needs the stored Jacobian%s");
  return by_dtype(ctx, [&](auto z) -> ngd_status {
    using T = decltype(z);
    if (theta) TRY(linearize<T>(ctx, theta));
    if (!ctx->lin_valid) return set_err(ctx, NGD_ERR_INVALID_ARG, "no linearization: pass theta%s");
    TRY(clear_status(ctx));
    TRY(form_gramian<T>(ctx, G, ldG));
    launch_lower_to_upper(G, ctx->p, ldG, ctx->stream);
    TRY(check_launch(ctx));
    return sync_status(ctx);
  });
}

ngd_status ngd_gramian_diag(ngd_ctx* ctx, const double* theta, double* d) {
  if (!ctx) return NGD_ERR_INVALID_ARG;
  if (!d) return set_err(ctx, NGD_ERR_INVALID_ARG, "d is NULL%s");
  return by_dtype(ctx, [&](auto z) -> ngd_status {
    using T = decltype(z);
    if (theta) TRY(linearize<T>(ctx, theta));
    if (!ctx->lin_valid) return set_err(ctx, NGD_ERR_INVALID_ARG, "no linearization: pass theta%s");
    return gram_diag_internal<T>(ctx, d);
  });
}

ngd_status ngd_nystrom_sketch_sampled(ngd_ctx* ctx, const double* theta, int ell, uint64_t seed, uint64_t step,
                                      int prec, int* idx, void* Omega, void* Y) {
  if (!ctx) return NGD_ERR_INVALID_ARG;
  if (!Omega || !Y || !idx) return set_err(ctx, NGD_ERR_INVALID_ARG, "idx/Omega/Y is NULL%s");
  if (ell < 1 || ell > std::min<int64_t>(ctx->p, 2048)) return set_err(ctx, NGD_ERR_INVALID_ARG, "ell out of range%s");
  if (!valid_prec(prec)) return set_err(ctx, NGD_ERR_INVALID_ARG, "bad sketch precision%s");
  if (ctx->dtype == NGD_F64 && prec != NGD_SKETCH_F64)
    return set_err(ctx, NGD_ERR_INVALID_ARG, "an F64 context sketches in F64 only%s");
  return by_dtype(ctx, [&](auto z) -> ngd_status {
    using T = decltype(z);
    if (theta) TRY(linearize<T>(ctx, theta));
    if (!ctx->lin_valid) return set_err(ctx, NGD_ERR_INVALID_ARG, "no linearization: pass theta%s");
    TRY(sketch_internal<T>(ctx, ell, seed, step, prec, 1));
    TRY(sync_status(ctx));
    const size_t w = (size_t)ctx->p * sizeof(T), sp = (size_t)ctx->ldP * sizeof(T);
    CK(cudaMemcpyAsync(idx, ctx->samp_idx, (size_t)ell * sizeof(int), cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpy2DAsync(Omega, w, ctx->Om, sp, w, ell, cudaMemcpyDeviceToDevice, ctx->stream));
    if (std::is_same<T, float>::value && acc64(prec))
      CK(cudaMemcpy2DAsync(Y, (size_t)ctx->p * 8, ctx->Y64, (size_t)ctx->ldP * 8, (size_t)ctx->p * 8, ell,
                           cudaMemcpyDeviceToDevice, ctx->stream));
    else
      CK(cudaMemcpy2DAsync(Y, w, ctx->Y, sp, w, ell, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return check_launch(ctx);
  });
}

ngd_status ngd_nystrom_factor(ngd_ctx* ctx, int ell, const void* Omega, const void* Y, int prec, double shift_scale,
                              void* U, double* lam, double* nu_out) {
  if (!ctx) return NGD_ERR_INVALID_ARG;
  if (!Omega || !Y || !U || !lam) return set_err(ctx, NGD_ERR_INVALID_ARG, "NULL argument%s");
  if (ell < 1 || ell > std::min<int64_t>(ctx->p, 2048)) return set_err(ctx, NGD_ERR_INVALID_ARG, "ell out of range%s");
  if (!valid_prec(prec) || !(shift_scale > 0.0)) return set_err(ctx, NGD_ERR_INVALID_ARG, "bad precision/shift%s");
  return by_dtype(ctx, [&](auto z) -> ngd_status {
    using T = decltype(z);
    TRY(ensure_ell(ctx, ell));
    const size_t w = (size_t)ctx->p * sizeof(T), sp = (size_t)ctx->ldP * sizeof(T);
    CK(cudaMemcpy2DAsync(ctx->Om, sp, Omega, w, w, ell, cudaMemcpyDeviceToDevice, ctx->stream));
    if (std::is_same<T, float>::value && acc64(prec))
      CK(cudaMemcpy2DAsync(ctx->Y64, (size_t)ctx->ldP * 8, Y, (size_t)ctx->p * 8, (size_t)ctx->p * 8, ell,
                           cudaMemcpyDeviceToDevice, ctx->stream));
    else
      CK(cudaMemcpy2DAsync(ctx->Y, sp, Y, w, w, ell, cudaMemcpyDeviceToDevice, ctx->stream));
    TRY(factor_internal<T>(ctx, ell, prec, shift_scale));
    if (std::is_same<T, float>::value && acc64(prec))
      CK(cudaMemcpy2DAsync(U, (size_t)ctx->p * 8, ctx->U64, (size_t)ctx->ldP * 8, (size_t)ctx->p * 8, ell,
                           cudaMemcpyDeviceToDevice, ctx->stream));
    else
      CK(cudaMemcpy2DAsync(U, w, ctx->U, sp, w, ell, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(lam, ctx->lam, ell * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    if (nu_out) {
      CK(cudaMemcpyAsync(ctx->h_scal + kSNu, ctx->scal + kSNu, 8, cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      *nu_out = ctx->h_scal[kSNu];
    }
    return check_launch(ctx);
  });
}

static bool valid_u_dtype(ngd_ctx* ctx, int u_dtype) {
  return u_dtype == NGD_F64 || (u_dtype == NGD_F32 && ctx->dtype == NGD_F32);
}

ngd_status ngd_precond_apply(ngd_ctx* ctx, int ell, const void* U, int u_dtype, const double* lam, double mu,
                             const double* v, double* zout) {
  if (!ctx) return NGD_ERR_INVALID_ARG;
  if (!U || !lam || !v || !zout || v == zout) return set_err(ctx, NGD_ERR_INVALID_ARG, "NULL or aliased argument%s");
  if (ell < 1 || ell > std::min<int64_t>(ctx->p, 2048) || !(mu >= 0.0))
    return set_err(ctx, NGD_ERR_INVALID_ARG, "ell/mu out of range%s");
  if (!valid_u_dtype(ctx, u_dtype)) return set_err(ctx, NGD_ERR_INVALID_ARG, "bad U dtype%s");
  TRY(ensure_ell(ctx, ell));
  precond(ctx, u_dtype == NGD_F64, U, ctx->p, ell, lam, mu, nullptr, v, zout, nullptr);
  return check_launch(ctx);
}

ngd_status ngd_pcg_solve(ngd_ctx* ctx, const double* theta, const double* g, double mu, const void* U, int u_dtype,
                         const double* lam, int ell, double rtol, int maxit, double* dout, int* iters, double* relres) {
  if (!ctx) return NGD_ERR_INVALID_ARG;
  if (!g || !dout || dout == g) return set_err(ctx, NGD_ERR_INVALID_ARG, "g/d NULL or aliased%s");
  if (!(mu > 0.0) || !(rtol >= 0.0) || maxit < 0) return set_err(ctx, NGD_ERR_INVALID_ARG, "mu/rtol/maxit%s");
  if (U && (ell < 1 || ell > std::min<int64_t>(ctx->p, 2048) || !lam || !valid_u_dtype(ctx, u_dtype)))
    return set_err(ctx, NGD_ERR_INVALID_ARG, "ell/lam/U dtype%s");
  return by_dtype(ctx, [&](auto z) -> ngd_status {
    using T = decltype(z);
    if (theta) TRY(linearize<T>(ctx, theta));
    if (!ctx->lin_valid) return set_err(ctx, NGD_ERR_INVALID_ARG, "no linearization: pass theta%s");
    if (U) TRY(ensure_ell(ctx, ell));
    return pcg_internal<T>(ctx, g, mu, nullptr, U, u_dtype == NGD_F64, ctx->p, lam, U ? ell : 0, rtol, maxit, dout,
                           iters, relres);
  });
}

ngd_status ngd_step(ngd_ctx* ctx, double* theta, const ngd_step_opts* o, ngd_step_info* info) {
  if (!ctx) return NGD_ERR_INVALID_ARG;
  if (!theta || !o) return set_err(ctx, NGD_ERR_INVALID_ARG, "theta/opts NULL%s");
  TRY(check_step_opts(ctx, o));
  return by_dtype(ctx, [&](auto z) -> ngd_status {
    using T = decltype(z);
    return step_impl<T>(ctx, theta, o, info);
  });
}

}  // extern "C"

// ------------------------------------------------------------------ batching form
// Many problems stepped together.  A batch step runs every problem's first stage (gradient,
// sketch, factor, damping), then the pCG solves, then every problem's line search.  Solves that
// fit the fused kernel are packed several to one cooperative launch: problem j gets a block group
// sized in proportion to its point count (at least the blocks its p and ell need), the groups
// synchronise on their own barrier counters, and the latency-bound phases of one solve overlap the
// row passes of the others.  How many solves share a launch is tuned on the batch itself: the
// first batch step times each feasible packing (1, 2, 4, 8 solves per launch) on its own
// launches and keeps the one with the lowest time per pCG iteration; the choice can be kept in a
// JSON file named by the environment variable NGD_AUTOTUNE_CACHE (key: SM count, p, padded
// Jacobian width, ell, problem count).
struct ngd_batch {
  std::vector<ngd_ctx*> ctx;
  std::string err;
  FusedPcgArgs* tab_host = nullptr;   // pinned: one table slot per problem and launch
  FusedPcgArgs* tab_dev = nullptr;
  unsigned int* bars = nullptr;       // one barrier counter (padded to 32 words) per problem
  int cap = 0;
  std::vector<int> last_iters;        // pCG iterations of each problem's previous solve
  int pack = 0;                       // solves per launch (0: not tuned yet)
  std::vector<int> tune_candidates;
  std::vector<double> tune_cost;      // ms per pCG iteration of each candidate
  std::string tune_key_base, tune_key;
  cudaEvent_t ev[2] = {};
  int launches_last = 0;              // cooperative launches of the last batch step's solves
};

namespace {

// JSON cache of tuned packings: a flat object {"key": value, ...}.
std::string tune_cache_path() {
  const char* p = std::getenv("NGD_AUTOTUNE_CACHE");
  return p ? std::string(p) : std::string();
}

int tune_cache_get(const std::string& key) {
  const std::string path = tune_cache_path();
  if (path.empty()) return 0;
  FILE* f = std::fopen(path.c_str(), "r");
  if (!f) return 0;
  std::string text;
  char buf[4096];
  size_t n;
  while ((n = std::fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, n);
  std::fclose(f);
  const std::string pat = "\"" + key + "\":";
  const size_t at = text.find(pat);
  if (at == std::string::npos) return 0;
  return std::atoi(text.c_str() + at + pat.size());
}

void tune_cache_put(const std::string& key, int value) {
  const std::string path = tune_cache_path();
  if (path.empty()) return;
  std::vector<std::pair<std::string, int>> entries;
  if (FILE* f = std::fopen(path.c_str(), "r")) {
    std::string text;
    char buf[4096];
    size_t n;
    while ((n = std::fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, n);
    std::fclose(f);
    size_t pos = 0;
    while ((pos = text.find('"', pos)) != std::string::npos) {
      const size_t end = text.find('"', pos + 1);
      if (end == std::string::npos) break;
      const size_t colon = text.find(':', end);
      if (colon == std::string::npos) break;
      entries.emplace_back(text.substr(pos + 1, end - pos - 1), std::atoi(text.c_str() + colon + 1));
      pos = colon + 1;
    }
  }
  bool found = false;
  for (auto& e : entries)
    if (e.first == key) {
      e.second = value;
      found = true;
    }
  if (!found) entries.emplace_back(key, value);
  const std::string tmp = path + ".tmp";
  FILE* f = std::fopen(tmp.c_str(), "w");
  if (!f) return;
  std::fprintf(f, "{");
  for (size_t i = 0; i < entries.size(); ++i)
    std::fprintf(f, "%s\n  \"%s\": %d", i ? "," : "", entries[i].first.c_str(), entries[i].second);
  std::fprintf(f, "\n}\n");
  std::fclose(f);
  std::rename(tmp.c_str(), path.c_str());
}

// Block groups of one launch: problems idx (their point counts N), at least gmin[k] blocks each,
// G blocks in all; the rest shared in proportion to N.  False if the minima do not fit.
bool split_blocks(const std::vector<int>& idx, const std::vector<ngd_ctx*>& ctx, const std::vector<int>& gmin, int G,
                  std::vector<int>& groups) {
  const size_t m = idx.size();
  groups.assign(m, 0);
  int need = 0;
  double ntot = 0.0;
  for (size_t k = 0; k < m; ++k) {
    need += gmin[k];
    ntot += (double)ctx[idx[k]]->N;
  }
  if (need > G) return false;
  int used = 0;
  for (size_t k = 0; k < m; ++k) {
    const int share = (int)std::floor((double)G * (double)ctx[idx[k]]->N / ntot);
    groups[k] = std::max(gmin[k], share);
    used += groups[k];
  }
  // trim the largest groups down to G, or hand the remainder to the largest problems
  while (used > G) {
    size_t best = m;
    for (size_t k = 0; k < m; ++k)
      if (groups[k] > gmin[k] && (best == m || groups[k] > groups[best])) best = k;
    if (best == m) return false;
    --groups[best];
    --used;
  }
  for (size_t k = 0; used < G; k = (k + 1) % m, ++used) ++groups[k];
  return true;
}

ngd_status batch_fail(ngd_batch* b, int i, ngd_status st) {
  b->err = "problem " + std::to_string(i) + ": " + ngd_last_error(b->ctx[(size_t)i]);
  return st;
}

// Packed launches for the solves `idxs` (in order), up to `want` solves per launch; table slots
// and barrier counters from *slot on.
ngd_status batch_launch(ngd_batch* b, const std::vector<int>& idxs, int want, std::vector<StepState>& st,
                        const ngd_step_opts* o, int* slot, int* launches) {
  ngd_ctx* ctx = b->ctx[0];            // CUDA failures of the shared stream are reported on problem 0
  const int G = fused_pcg_blocks();
  cudaStream_t s = ctx->stream;
  size_t pos = 0;
  while (pos < idxs.size()) {
    // take up to `want` solves whose minimum block groups fit the GPU together
    std::vector<int> idx, gmin, groups;
    while (pos < idxs.size() && (int)idx.size() < want) {
      const int i = idxs[pos];
      ngd_ctx* c = b->ctx[(size_t)i];
      const int gm = fused_pcg_min_blocks(c->p, st[(size_t)i].ell_pc);
      std::vector<int> trial(idx), tmin(gmin);
      trial.push_back(i);
      tmin.push_back(gm);
      if (!split_blocks(trial, b->ctx, tmin, G, groups)) break;
      idx.push_back(i);
      gmin.push_back(gm);
      ++pos;
    }
    if (idx.empty()) return NGD_ERR_UNSUPPORTED;          // cannot happen: one solve takes all blocks
    split_blocks(idx, b->ctx, gmin, G, groups);
    int gb0 = 0;
    for (size_t k = 0; k < idx.size(); ++k) {
      const int i = idx[k];
      ngd_ctx* c = b->ctx[(size_t)i];
      StepState& ss = st[(size_t)i];
      TRY(pcg_begin(c, o->rtol, o->maxit));
      FusedPcgArgs fa;
      if (!fused_args<float>(c, c->g, 0.0, c->scal + kSMu, ss.Ust, ss.u_f64, c->ldP, c->lam, ss.ell_pc, c->d,
                             groups[k], &fa))
        return set_err(c, NGD_ERR_UNSUPPORTED, "fused solve unavailable in the batch%s");
      fa.gb0 = gb0;
      fa.gG = groups[k];
      fa.bar = b->bars + (size_t)(*slot + (int)k) * 32;
      b->tab_host[*slot + (int)k] = fa;
      gb0 += groups[k];
    }
    const int m = (int)idx.size();
    if (cudaMemsetAsync(b->bars + (size_t)*slot * 32, 0, (size_t)m * 32 * sizeof(unsigned), s) != cudaSuccess ||
        cudaMemcpyAsync(b->tab_dev + *slot, b->tab_host + *slot, (size_t)m * sizeof(FusedPcgArgs),
                        cudaMemcpyHostToDevice, s) != cudaSuccess)
      return batch_fail(b, idx[0], set_err(b->ctx[(size_t)idx[0]], NGD_ERR_CUDA, "batch solve table%s"));
    const cudaError_t e = launch_pcg_fused_multi(b->tab_dev + *slot, b->tab_host + *slot, m, s);
    if (e != cudaSuccess)
      return batch_fail(b, idx[0], set_err(b->ctx[(size_t)idx[0]], NGD_ERR_CUDA, "multi-problem solve: %s",
                                           cudaGetErrorString(e)));
    ++*launches;
    *slot += m;
  }
  return NGD_OK;
}

// The pCG solves of the problems in `solve` (stage 2 of a batch step), packed b->pack to a
// cooperative launch.  Untuned, the step first gives every candidate packing the same number of
// solves (consecutive ones in the order below), times them as a whole, and keeps the candidate with
// the least time per pCG iteration for the remaining solves and the later steps.
ngd_status batch_solves(ngd_batch* b, const std::vector<int>& solve, std::vector<StepState>& st,
                        const ngd_step_opts* o) {
  ngd_ctx* ctx = b->ctx[0];
  cudaStream_t s = ctx->stream;
  // order: longest previous solves first, so that a launch holds solves of similar length
  std::vector<int> order(solve);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->last_iters[x] > b->last_iters[y]; });
  int slot = 0, launches = 0;
  size_t pos = 0;
  if (b->pack == 0) {
    const size_t nc = b->tune_candidates.size();
    const size_t span = std::max<size_t>(1, std::min<size_t>(8, order.size() / nc));
    for (size_t c = 0; c < nc && pos + span <= order.size(); ++c, pos += span) {
      std::vector<int> seg(order.begin() + (long)pos, order.begin() + (long)(pos + span));
      CK(cudaEventRecord(b->ev[0], s));
      TRY(batch_launch(b, seg, b->tune_candidates[c], st, o, &slot, &launches));
      CK(cudaEventRecord(b->ev[1], s));
      for (int i : seg) {
        ngd_ctx* c2 = b->ctx[(size_t)i];
        CK(cudaMemcpyAsync(c2->h_pcg, c2->pcg, sizeof(PcgScalars), cudaMemcpyDeviceToHost, s));
      }
      CK(cudaStreamSynchronize(s));
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]);
      long iters = 0;
      for (int i : seg) iters += b->ctx[(size_t)i]->h_pcg->iters;
      b->tune_cost[c] = iters > 0 ? ms / (double)iters : 1e30;
    }
    size_t best = 0;
    for (size_t k = 1; k < b->tune_cost.size(); ++k)
      if (b->tune_cost[k] >= 0.0 && (b->tune_cost[best] < 0.0 || b->tune_cost[k] < b->tune_cost[best])) best = k;
    b->pack = b->tune_candidates[best];
    if (b->tune_cost[best] >= 0.0) tune_cache_put(b->tune_key, b->pack);
  }
  std::vector<int> rest(order.begin() + (long)pos, order.end());
  TRY(batch_launch(b, rest, b->pack, st, o, &slot, &launches));
  b->launches_last = launches;
  for (int i : solve) {
    ngd_ctx* c = b->ctx[(size_t)i];
    CK(cudaMemcpyAsync(c->h_pcg, c->pcg, sizeof(PcgScalars), cudaMemcpyDeviceToHost, s));
  }
  CK(cudaStreamSynchronize(s));
  for (int i : solve) {
    ngd_ctx* c = b->ctx[(size_t)i];
    if (c->h_pcg->status & kStatTimeout) return batch_fail(b, i, set_err(c, NGD_ERR_TIMEOUT, "solve barrier timed out%s"));
    const ngd_status r = pcg_result(c, c->h_pcg, &st[(size_t)i].iters, &st[(size_t)i].relres);
    if (r != NGD_OK) return batch_fail(b, i, r);
    CK(cudaEventRecord(c->ev[4], c->stream));
    b->last_iters[(size_t)i] = st[(size_t)i].iters;
  }
  return NGD_OK;
}

}  // namespace

extern "C" {

ngd_status ngd_batch_create(const ngd_problem_desc* descs, int n, ngd_batch** out) {
  if (!out) return NGD_ERR_INVALID_ARG;
  *out = nullptr;
  if (!descs || n < 1) return NGD_ERR_INVALID_ARG;
  ngd_batch* b = new (std::nothrow) ngd_batch;
  if (!b) return NGD_ERR_OOM;
  for (int i = 0; i < n; ++i) {
    ngd_problem_desc d = descs[i];
    d.stream = descs[0].stream;
    ngd_ctx* c = nullptr;
    const ngd_status st = ngd_create(&d, &c);
    if (st != NGD_OK) {
      ngd_batch_destroy(b);
      return st;
    }
    b->ctx.push_back(c);
  }
  b->cap = n;
  b->last_iters.assign((size_t)n, 0);
  if (cudaMallocHost((void**)&b->tab_host, (size_t)n * sizeof(FusedPcgArgs)) != cudaSuccess ||
      cudaMalloc((void**)&b->tab_dev, (size_t)n * sizeof(FusedPcgArgs)) != cudaSuccess ||
      cudaMalloc((void**)&b->bars, (size_t)n * 32 * sizeof(unsigned)) != cudaSuccess ||
      cudaEventCreate(&b->ev[0]) != cudaSuccess || cudaEventCreate(&b->ev[1]) != cudaSuccess) {
    cudaGetLastError();
    ngd_batch_destroy(b);
    return NGD_ERR_OOM;
  }
  // packings to try (2^k solves per launch while their minimum block groups fit the GPU)
  const ngd_ctx* c0 = b->ctx[0];
  b->tune_candidates = {1};
  for (int k = 2; k <= 8 && k <= n; k *= 2) b->tune_candidates.push_back(k);
  b->tune_cost.assign(b->tune_candidates.size(), -1.0);
  int nsm = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  b->tune_key_base = "sm" + std::to_string(nsm) + "_p" + std::to_string(c0->p) + "_ldJ" + std::to_string(c0->ldJ) +
                     "_n" + std::to_string(n);
  *out = b;
  return NGD_OK;
}

void ngd_batch_destroy(ngd_batch* b) {
  if (!b) return;
  for (ngd_ctx* c : b->ctx) ngd_destroy(c);
  if (b->tab_host) cudaFreeHost(b->tab_host);
  if (b->tab_dev) cudaFree(b->tab_dev);
  if (b->bars) cudaFree(b->bars);
  for (auto& e : b->ev)
    if (e) cudaEventDestroy(e);
  delete b;
}

int ngd_batch_size(const ngd_batch* b) { return b ? (int)b->ctx.size() : 0; }

ngd_ctx* ngd_batch_context(ngd_batch* b, int i) {
  if (!b || i < 0 || i >= (int)b->ctx.size()) return nullptr;
  return b->ctx[i];
}

const char* ngd_batch_last_error(const ngd_batch* b) { return b ? b->err.c_str() : ""; }

ngd_status ngd_batch_set_packing(ngd_batch* b, int solves_per_launch) {
  if (!b || solves_per_launch < 0 || solves_per_launch > 64) return NGD_ERR_INVALID_ARG;
  b->pack = solves_per_launch;
  if (solves_per_launch == 0) std::fill(b->tune_cost.begin(), b->tune_cost.end(), -1.0);
  return NGD_OK;
}

int ngd_batch_packing(const ngd_batch* b) { return b ? b->pack : -1; }

int ngd_batch_solve_launches(const ngd_batch* b) { return b ? b->launches_last : -1; }

ngd_status ngd_batch_step(ngd_batch* b, double* const* thetas, const ngd_step_opts* opts, ngd_step_info* infos) {
  if (!b) return NGD_ERR_INVALID_ARG;
  if (!thetas || !opts) {
    b->err = "thetas/opts NULL";
    return NGD_ERR_INVALID_ARG;
  }
  b->err.clear();
  const size_t n = b->ctx.size();
  b->tune_key = b->tune_key_base + "_ell" + std::to_string(opts->ell);
  if (b->pack == 0) {
    const int cached = tune_cache_get(b->tune_key);
    if (cached > 0) b->pack = cached;
  }
  std::vector<ngd_step_opts> o(n, *opts);
  for (size_t i = 0; i < n; ++i) {
    o[i].seed = opts->seed + i;
    const ngd_status v = check_step_opts(b->ctx[i], &o[i]);
    if (v != NGD_OK) return batch_fail(b, (int)i, v);
  }
  std::vector<StepState> st(n);
  // stage 1 for every problem
  for (size_t i = 0; i < n; ++i) {
    ngd_ctx* c = b->ctx[i];
    const ngd_status r = by_dtype(c, [&](auto z) -> ngd_status {
      using T = decltype(z);
      return step_prepare<T>(c, thetas[i], &o[i], st[i]);
    });
    if (r != NGD_OK) return batch_fail(b, (int)i, r);
  }
  // stage 2: the fused solves packed several to a launch (a single problem, or a packing of one,
  // keeps the whole-grid launch), the others one by one
  std::vector<int> packed;
  for (size_t i = 0; i < n; ++i) {
    ngd_ctx* c = b->ctx[i];
    const bool pre = st[i].Ust != nullptr && st[i].ell_pc > 0;
    if (n > 1 && b->pack != 1 && !st[i].full && c->dtype == NGD_F32 && c->stored_j && c->yph &&
        fused_pcg_supported(c->p, c->ldJ, pre ? st[i].ell_pc : 0) &&
        fused_pcg_slots(c->ldJ) == fused_pcg_slots(b->ctx[0]->ldJ))
      packed.push_back((int)i);
  }
  if (packed.size() < 2) packed.clear();
  std::vector<char> is_packed(n, 0);
  for (int i : packed) is_packed[(size_t)i] = 1;
  for (size_t i = 0; i < n; ++i) {
    if (is_packed[i]) continue;
    ngd_ctx* c = b->ctx[i];
    const ngd_status r = by_dtype(c, [&](auto z) -> ngd_status {
      using T = decltype(z);
      return step_solve<T>(c, &o[i], st[i]);
    });
    if (r != NGD_OK) return batch_fail(b, (int)i, r);
    b->last_iters[i] = st[i].iters;
  }
  if (!packed.empty()) {
    const ngd_status r = batch_solves(b, packed, st, opts);
    if (r != NGD_OK) return r;
  }
  // stage 3 for every problem
  for (size_t i = 0; i < n; ++i) {
    ngd_ctx* c = b->ctx[i];
    const ngd_status r = by_dtype(c, [&](auto z) -> ngd_status {
      using T = decltype(z);
      return step_finish<T>(c, thetas[i], &o[i], st[i], infos ? infos + i : nullptr);
    });
    if (r != NGD_OK) return batch_fail(b, (int)i, r);
  }
  return NGD_OK;
}

}  // extern "C"
