// Internal declarations shared by the CUDA translation units of libngd.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ngd.h"

namespace ngd {

constexpr int kMaxLayers = 8;    // affine layers
constexpr int kMaxD = 16;        // input dimension
constexpr int kMaxWidth = 512;   // hidden width
constexpr int kThreads = 256;    // block size of the Taylor-mode kernels

// Device status bits (the status word lives in device memory; the host maps a
// set bit to an ngd_status at the next synchronising call).
enum : int {
  kStatNotSpd = 1,
  kStatBreakdown = 2,
  kStatNonFinite = 4,
  kStatTimeout = 8,
  kStatSample = 16,      // fewer positive diagonal entries of G than the sample size
  kStatDrain = 32,       // after a timeout, waiting for work already issued ran out as well
};

// Network description passed by value to the kernels.
struct NetDesc {
  int n_layers;                    // affine layers L+1
  int d;                           // input dimension
  int C;                           // Taylor channels per point: value, d gradient entries, Laplacian
  int pde;                         // ngd_pde
  double kappa;
  int max_width;                   // max over layers of widths[l] for l = 0..n_layers-1 (inputs of affine layers)
  int width[kMaxLayers + 1];
  int64_t theta_off[kMaxLayers];   // W_l starts here in theta; b_l follows after n_out*n_in
  int64_t wt_off[kMaxLayers];      // transposed W_l (n_in x n_out) in the prepared buffer
  int64_t wr_off[kMaxLayers];      // row-major W_l (n_out x n_in) in the prepared buffer
  int64_t b_off[kMaxLayers];       // b_l in the prepared buffer
  int64_t p;                       // number of parameters
  int64_t prep_size;               // elements of the prepared buffer (2p)
  int64_t tape_per_point;          // C * sum of hidden widths (stored Taylor coefficients per point)
};

// Count of kernel launches made by the library (process-wide, for instrumentation).
void note_launch(int n = 1);

// Problem data on the device (caller-owned arrays) and the point range processed.
struct PointSet {
  const double* X;       // N x d
  const double* target;  // N
  const double* w;       // N
  int64_t n_int;
  int64_t N;
};

// ---------------------------------------------------------------- taylor.cu
// theta (float64) -> prepared per-layer weights in the working dtype:
// transposed W (for the forward), row-major W (for the reverse) and biases.
template <typename T>
void launch_prep_weights(const NetDesc& net, const double* theta, T* prep, cudaStream_t s);

// Shared-memory bytes per point of each Taylor kernel.
size_t fwd_smem_per_point(const NetDesc& net, size_t elt);
size_t jac_smem_per_point(const NetDesc& net, size_t elt);
size_t jvp_smem_per_point(const NetDesc& net, size_t elt);

// Residuals r (nullable) and per-block loss partials for rows [row0, row0+nrows).
// tape (nullable): store the Taylor coefficients (t, grad a, Delta a per hidden layer).
template <typename T>
// chan (nullable): the C = d + 2 output channels (u, grad u, Delta u) of each point as float64,
// chan[row * C + c].
int launch_forward(const NetDesc& net, const PointSet& ps, const T* prep, int64_t row0, int64_t nrows,
                   double* r, double* loss_part, T* tape, int tp, cudaStream_t s, double* chan = nullptr);

// Jacobian rows J[row - row0, :] (row stride ldJ) for rows [row0, row0+nrows), plus r and
// loss partials (when not from_tape).  tape_in non-null: reverse pass from stored coefficients.
template <typename T>
int launch_jacobian(const NetDesc& net, const PointSet& ps, const T* prep, int64_t row0, int64_t nrows,
                    T* J, int64_t ldJ, double* r, double* loss_part, const T* tape_in, int tp, cudaStream_t s);

// Jv for all rows (forward-mode tangents); prep_t = prepared tangent weights of v.
template <typename T>
int launch_jvp(const NetDesc& net, const PointSet& ps, const T* prep, const T* prep_t, double* out,
               int tp, cudaStream_t s);

// ---------------------------------------------------------------- vjp_rev.cu
// Reverse pass by layers over the points [row0, row0 + npts) (buffers [pt * C + c][ldb]); tape
// row-indexed (tape + row * tape_per_point), toff the hidden layer's offset in a point's tape.
template <typename T>
void launch_rev_seed(const NetDesc& net, const PointSet& ps, int64_t row0, int64_t npts, const double* cot, T* A,
                     int ldb, cudaStream_t s);
template <typename T>
void launch_rev_input(const NetDesc& net, const PointSet& ps, int l, const T* tape, int64_t toff, int64_t row0,
                      int64_t npts, T* X, int ldb, cudaStream_t s);
template <typename T>
void launch_rev_tanh(const NetDesc& net, int lh, const T* tape, int64_t toff, int64_t row0, int64_t npts,
                     const T* Xb, T* A, int ldb, cudaStream_t s);
void launch_rev_sum(const double* part, int nz, int64_t stride, int64_t n, double* out, int accumulate,
                    cudaStream_t s);
// forward tangents by layers (J v): tanh tangent of hidden layer lh, and J v from the output tangents
template <typename T>
void launch_fwd_tangent(const NetDesc& net, int lh, const T* tape, int64_t toff, int64_t row0, int64_t npts,
                        const T* Ad, const T* bdot, T* Xd, int ldb, cudaStream_t s);
template <typename T>
void launch_jvp_out(const NetDesc& net, const PointSet& ps, int64_t row0, int64_t npts, const T* Ad, const T* bdot,
                    int ldb, double* out, cudaStream_t s);

}  // namespace ngd
