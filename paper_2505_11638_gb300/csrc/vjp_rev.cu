// Matrix-free vector-Jacobian product J^T c by the reverse of the Taylor-mode forward, layer by
// layer over all points of a chunk (Thm. 1: the Gramian is J^T W J; Sec. 4.1.2 "recompute batch
// Jacobian on the fly" without forming its rows).
//
// For one point, the hidden layer l maps the C = d + 2 channels (value, gradient, Laplacian) of
// its input x_{l-1} to a_l = W_l x_{l-1} + b_l (every channel; b_l enters the value channel only)
// and then through tanh (Taylor-mode rule, see taylor.cu).  The reverse of the whole forward for
// the cotangent c_r of the residual r_r seeds the output channels with c_r times the residual's
// coefficients and walks back:
//   W_bar_l += sum over points and channels of abar_l (outer) x_{l-1},  b_bar_l += sum of abar_l
//   (value channel),  xbar_{l-1} = W_l^T abar_l,  abar_{l-1} = adjoint of tanh (channel mixing
//   within the point, from the stored t, grad a, Delta a).
// With the points' channels as the rows of [k = pt C + c][neuron] buffers, W_bar_l is one GEMM
// with K = (points) x C and xbar_{l-1} another (the same arithmetic as the Jacobian kernel's rows
// summed over points, without writing N x p entries).  This file holds the elementwise kernels;
// the GEMMs are the library's SIMT GEMM (FP32 sums folded into FP64 every 128 terms, FP64 K-slice
// partials added in a fixed order).
#include <cuda_runtime.h>

#include <algorithm>

#include "ngd_internal.cuh"

namespace ngd {

namespace {

__device__ __forceinline__ bool spatial(const NetDesc& net, int k) { return !(net.pde == NGD_PDE_HEAT && k == 0); }

// Seeds of the output layer (n_out = 1): the coefficients of r in (u, grad u, Delta u) times c_r.
template <typename T>
__global__ void k_rev_seed(NetDesc net, PointSet ps, int64_t row0, int64_t npts, const double* __restrict__ cot,
                           T* __restrict__ A, int ldb) {
  const int C = net.C, d = net.d;
  const int64_t total = npts * C;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += st) {
    const int64_t pt = e / C;
    const int c = (int)(e - pt * C);
    const int64_t row = row0 + pt;
    const double cr = cot[row];
    double v = 0.0;
    if (row < ps.n_int) {
      if (net.pde == NGD_PDE_HEAT)
        v = c == 1 ? cr : (c == d + 1 ? -net.kappa * cr : 0.0);
      else
        v = c == d + 1 ? cr : 0.0;
    } else {
      v = c == 0 ? cr : 0.0;
    }
    A[e * ldb] = (T)v;
  }
}

// Input channels x_{l-1} of affine layer l for the chunk's points: for l >= 1 from the tape of
// hidden layer l - 1 (t, grad a, Delta a -> t, s1 grad a, s1 Delta a + s2 q); for l = 0 the point
// itself (x, grad x = I, Delta x = 0).  tape: row-indexed (tape + row * tpp).
template <typename T>
__global__ void k_rev_input(NetDesc net, PointSet ps, int l, const T* __restrict__ tape, int64_t toff,
                            int64_t row0, int64_t npts, T* __restrict__ X, int ldb) {
  const int C = net.C, d = net.d, n_in = net.width[l];
  const int64_t total = npts * n_in;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += st) {
    const int64_t pt = e / n_in;
    const int j = (int)(e - pt * n_in);
    const int64_t row = row0 + pt;
    T* xo = X + pt * C * ldb + j;
    if (l == 0) {
      xo[0] = (T)ps.X[row * d + j];
      for (int k = 0; k < d; ++k) xo[(int64_t)(1 + k) * ldb] = k == j ? T(1) : T(0);
      xo[(int64_t)(d + 1) * ldb] = T(0);
    } else {
      const T* tp = tape + row * net.tape_per_point + toff + j;
      const T t = tp[0];
      const T s1 = T(1) - t * t, s2 = T(-2) * t * s1;
      T qs = T(0);
      for (int k = 0; k < d; ++k) {
        const T ga = tp[(int64_t)(1 + k) * n_in];
        if (spatial(net, k)) qs += ga * ga;
        xo[(int64_t)(1 + k) * ldb] = s1 * ga;
      }
      xo[0] = t;
      xo[(int64_t)(d + 1) * ldb] = s1 * tp[(int64_t)(d + 1) * n_in] + s2 * qs;
    }
  }
}

// Adjoint through tanh of hidden layer lh (width nh): abar from xbar and the stored coefficients,
//   abar        = s1 xbar + s2 sum_k grad_k a grad_k xbar + (s2 Delta a + s3 q) Delta xbar
//   grad_k abar = s1 grad_k xbar + 2 s2 grad_k a Delta xbar   (k spatial; s1 grad_k xbar otherwise)
//   Delta abar  = s1 Delta xbar
template <typename T>
__global__ void k_rev_tanh(NetDesc net, int lh, const T* __restrict__ tape, int64_t toff, int64_t row0, int64_t npts,
                           const T* __restrict__ Xb, T* __restrict__ A, int ldb) {
  const int C = net.C, d = net.d, nh = net.width[lh + 1];
  const int64_t total = npts * nh;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += st) {
    const int64_t pt = e / nh;
    const int j = (int)(e - pt * nh);
    const T* tp = tape + (row0 + pt) * net.tape_per_point + toff + j;
    const T t = tp[0];
    const T s1 = T(1) - t * t, s2 = T(-2) * t * s1, s3 = T(-2) * s1 * (T(1) - T(3) * t * t);
    const T la = tp[(int64_t)(d + 1) * nh];
    const T* xb = Xb + pt * C * ldb + j;
    const T xbl = xb[(int64_t)(d + 1) * ldb];
    T qs = T(0), sg = T(0);
    for (int k = 0; k < d; ++k) {
      const T ga = tp[(int64_t)(1 + k) * nh];
      if (spatial(net, k)) qs += ga * ga;
      sg += ga * xb[(int64_t)(1 + k) * ldb];
    }
    T* a = A + pt * C * ldb + j;
    a[0] = s1 * xb[0] + s2 * sg + (s2 * la + s3 * qs) * xbl;
    for (int k = 0; k < d; ++k) {
      const T ga = tp[(int64_t)(1 + k) * nh];
      a[(int64_t)(1 + k) * ldb] = s1 * xb[(int64_t)(1 + k) * ldb] + (spatial(net, k) ? T(2) * s2 * ga * xbl : T(0));
    }
    a[(int64_t)(d + 1) * ldb] = s1 * xbl;
  }
}

// Forward tangents through tanh of hidden layer lh (width nh): from the tangent adot of the
// pre-activation channels (the bias tangent bdot added to the value channel) and the stored
// coefficients, the tangent xdot of the layer's output channels:
//   xdot        = s1 adot
//   grad_k xdot = s1 grad_k adot + s2 adot grad_k a
//   Delta xdot  = s1 Delta adot + s2 (adot Delta a + 2 sum_k spatial grad_k a grad_k adot) + s3 adot q
template <typename T>
__global__ void k_fwd_tangent(NetDesc net, int lh, const T* __restrict__ tape, int64_t toff, int64_t row0,
                              int64_t npts, const T* __restrict__ Ad, const T* __restrict__ bdot,
                              T* __restrict__ Xd, int ldb) {
  const int C = net.C, d = net.d, nh = net.width[lh + 1];
  const int64_t total = npts * nh;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += st) {
    const int64_t pt = e / nh;
    const int j = (int)(e - pt * nh);
    const T* tp = tape + (row0 + pt) * net.tape_per_point + toff + j;
    const T t = tp[0];
    const T s1 = T(1) - t * t, s2 = T(-2) * t * s1, s3 = T(-2) * s1 * (T(1) - T(3) * t * t);
    const T* ad = Ad + pt * C * ldb + j;
    const T a0 = ad[0] + bdot[j];
    T qs = T(0), qd = T(0);
    T* xd = Xd + pt * C * ldb + j;
    for (int k = 0; k < d; ++k) {
      const T ga = tp[(int64_t)(1 + k) * nh];
      const T gad = ad[(int64_t)(1 + k) * ldb];
      if (spatial(net, k)) {
        qs += ga * ga;
        qd += ga * gad;
      }
      xd[(int64_t)(1 + k) * ldb] = s1 * gad + s2 * a0 * ga;
    }
    const T la = tp[(int64_t)(d + 1) * nh];
    xd[0] = s1 * a0;
    xd[(int64_t)(d + 1) * ldb] = s1 * ad[(int64_t)(d + 1) * ldb] + s2 * (a0 * la + T(2) * qd) + s3 * a0 * qs;
  }
}

// J v of each point from the tangents of the output channels (the output bias tangent added to
// the value channel): the residual's coefficients in (u, grad u, Delta u).
template <typename T>
__global__ void k_jvp_out(NetDesc net, PointSet ps, int64_t row0, int64_t npts, const T* __restrict__ Ad,
                          const T* __restrict__ bdot, int ldb, double* __restrict__ out) {
  const int C = net.C, d = net.d;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t pt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pt < npts; pt += st) {
    const T* ad = Ad + pt * C * ldb;
    const int64_t row = row0 + pt;
    double v;
    if (row < ps.n_int)
      v = net.pde == NGD_PDE_HEAT ? (double)ad[ldb] - net.kappa * (double)ad[(int64_t)(d + 1) * ldb]
                                  : (double)ad[(int64_t)(d + 1) * ldb];
    else
      v = (double)ad[0] + (double)bdot[0];
    out[row] = v;
  }
}

// out[i] (+)= sum over the nz K-slice partials part[z * stride + i], in slice order.
__global__ void k_rev_sum(const double* __restrict__ part, int nz, int64_t stride, int64_t n, double* __restrict__ out,
                          int accumulate) {
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += st) {
    double s = accumulate ? out[i] : 0.0;
    for (int z = 0; z < nz; ++z) s += part[z * stride + i];
    out[i] = s;
  }
}

int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8192)); }

}  // namespace

template <typename T>
void launch_rev_seed(const NetDesc& net, const PointSet& ps, int64_t row0, int64_t npts, const double* cot, T* A,
                     int ldb, cudaStream_t s) {
  k_rev_seed<T><<<grid_for(npts * net.C), 256, 0, s>>>(net, ps, row0, npts, cot, A, ldb);
  note_launch();
}
template <typename T>
void launch_rev_input(const NetDesc& net, const PointSet& ps, int l, const T* tape, int64_t toff, int64_t row0,
                      int64_t npts, T* X, int ldb, cudaStream_t s) {
  k_rev_input<T><<<grid_for(npts * net.width[l]), 256, 0, s>>>(net, ps, l, tape, toff, row0, npts, X, ldb);
  note_launch();
}
template <typename T>
void launch_rev_tanh(const NetDesc& net, int lh, const T* tape, int64_t toff, int64_t row0, int64_t npts,
                     const T* Xb, T* A, int ldb, cudaStream_t s) {
  k_rev_tanh<T><<<grid_for(npts * net.width[lh + 1]), 256, 0, s>>>(net, lh, tape, toff, row0, npts, Xb, A, ldb);
  note_launch();
}
template <typename T>
void launch_fwd_tangent(const NetDesc& net, int lh, const T* tape, int64_t toff, int64_t row0, int64_t npts,
                        const T* Ad, const T* bdot, T* Xd, int ldb, cudaStream_t s) {
  k_fwd_tangent<T><<<grid_for(npts * net.width[lh + 1]), 256, 0, s>>>(net, lh, tape, toff, row0, npts, Ad, bdot, Xd,
                                                                       ldb);
  note_launch();
}
template <typename T>
void launch_jvp_out(const NetDesc& net, const PointSet& ps, int64_t row0, int64_t npts, const T* Ad, const T* bdot,
                    int ldb, double* out, cudaStream_t s) {
  k_jvp_out<T><<<grid_for(npts), 256, 0, s>>>(net, ps, row0, npts, Ad, bdot, ldb, out);
  note_launch();
}
template void launch_fwd_tangent<float>(const NetDesc&, int, const float*, int64_t, int64_t, int64_t, const float*,
                                        const float*, float*, int, cudaStream_t);
template void launch_fwd_tangent<double>(const NetDesc&, int, const double*, int64_t, int64_t, int64_t, const double*,
                                         const double*, double*, int, cudaStream_t);
template void launch_jvp_out<float>(const NetDesc&, const PointSet&, int64_t, int64_t, const float*, const float*, int,
                                    double*, cudaStream_t);
template void launch_jvp_out<double>(const NetDesc&, const PointSet&, int64_t, int64_t, const double*, const double*,
                                     int, double*, cudaStream_t);

void launch_rev_sum(const double* part, int nz, int64_t stride, int64_t n, double* out, int accumulate,
                    cudaStream_t s) {
  k_rev_sum<<<grid_for(n), 256, 0, s>>>(part, nz, stride, n, out, accumulate);
  note_launch();
}

template void launch_rev_seed<float>(const NetDesc&, const PointSet&, int64_t, int64_t, const double*, float*, int,
                                     cudaStream_t);
template void launch_rev_seed<double>(const NetDesc&, const PointSet&, int64_t, int64_t, const double*, double*, int,
                                      cudaStream_t);
template void launch_rev_input<float>(const NetDesc&, const PointSet&, int, const float*, int64_t, int64_t, int64_t,
                                      float*, int, cudaStream_t);
template void launch_rev_input<double>(const NetDesc&, const PointSet&, int, const double*, int64_t, int64_t, int64_t,
                                       double*, int, cudaStream_t);
template void launch_rev_tanh<float>(const NetDesc&, int, const float*, int64_t, int64_t, int64_t, const float*,
                                     float*, int, cudaStream_t);
template void launch_rev_tanh<double>(const NetDesc&, int, const double*, int64_t, int64_t, int64_t, const double*,
                                      double*, int, cudaStream_t);

}  // namespace ngd
