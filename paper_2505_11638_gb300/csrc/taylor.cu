// Taylor-mode (forward-Laplacian) kernels of the tanh MLP: residuals, Jacobian rows
// (the hand-written reverse pass) and Jacobian-vector products (forward tangents).
//
// Network (Sec. 2.3): x_l = tanh(W_l x_{l-1} + b_l) for the hidden layers, u = W x + b at
// the output.  Each point carries C = d + 2 channels: value, the d entries of the
// gradient and the (spatial) Laplacian.  Through a hidden layer, with a = W x + b,
// t = tanh a, s1 = 1 - t^2, s2 = -2 t s1, s3 = -2 s1 (1 - 3 t^2), q = sum_{k spatial} (grad_k a)^2:
//   x' = t,  grad x' = s1 grad a,  Delta x' = s1 Delta a + s2 q.
// Residual rows (Sec. 2.2.1, Eq. energy_poisson): Poisson interior r = Delta u + f, heat
// interior r = u_t - kappa Delta u - f (coordinate 0 is t and is excluded from q), boundary
// r = u - g.  J[r, :] = grad_theta r_r is the Jacobian of Thm. 1 (Eq. G_matrixfree).
//
// GB300 mapping: one CTA owns a tile of TP points and keeps every channel of those
// points in shared memory across all layers, so the cross-channel sum q of the
// epilogue never leaves the thread that owns (point, neuron).  Weights are read from a
// per-step prepared copy (working dtype, transposed for the forward, row-major for the
// reverse) that stays L1/L2 resident.  The reverse pass recomputes the forward
// coefficients in shared memory (or reloads them from a stored tape) and writes each
// Jacobian row segment with coalesced stores.
#include <cuda_runtime.h>

#include <algorithm>

#include "ngd_internal.cuh"

namespace ngd {

template <typename T> __device__ __forceinline__ T tanh_t(T x);
template <> __device__ __forceinline__ float tanh_t<float>(float x) { return tanhf(x); }
template <> __device__ __forceinline__ double tanh_t<double>(double x) { return tanh(x); }

template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ bool is_spatial(const NetDesc& net, int k) {  // k = gradient index 0..d-1
  return !(net.pde == NGD_PDE_HEAT && k == 0);
}

// ---------------------------------------------------------------------------- prep
template <typename T>
__global__ void k_prep(NetDesc net, const double* __restrict__ theta, T* __restrict__ prep) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < net.p; k += stride) {
    int l = 0;
    while (l + 1 < net.n_layers && k >= net.theta_off[l + 1]) ++l;
    const int64_t local = k - net.theta_off[l];
    const int n_in = net.width[l], n_out = net.width[l + 1];
    const T v = (T)theta[k];
    if (local < (int64_t)n_out * n_in) {
      const int i = (int)(local / n_in), j = (int)(local - (int64_t)i * n_in);
      prep[net.wr_off[l] + local] = v;
      prep[net.wt_off[l] + (int64_t)j * n_out + i] = v;
    } else {
      prep[net.b_off[l] + (local - (int64_t)n_out * n_in)] = v;
    }
  }
}

template <typename T>
void launch_prep_weights(const NetDesc& net, const double* theta, T* prep, cudaStream_t s) {
  const int threads = 256;
  const int blocks = (int)std::min<int64_t>((net.p + threads - 1) / threads, 4096);
  k_prep<T><<<blocks, threads, 0, s>>>(net, theta, prep); note_launch();
}
template void launch_prep_weights<float>(const NetDesc&, const double*, float*, cudaStream_t);
template void launch_prep_weights<double>(const NetDesc&, const double*, double*, cudaStream_t);

// ---------------------------------------------------------------------------- forward pieces
// One hidden layer l for the points [0, npts) of the tile: in/out are [pt][C][maxw] buffers
// (per-point stride pstride).  Layer 0 reads the points from global memory and uses
// grad x_0 = I, Delta x_0 = 0.  tape (smem or global, nullable): t, grad a, Delta a as
// [C][n_out] per point at offset tape_off.
template <typename T, int MAXC, int PP>
__device__ __forceinline__ void fwd_hidden(const NetDesc& net, int l, const T* __restrict__ prep,
                                           const double* __restrict__ X, int64_t row0, int npts,
                                           const T* in, T* out, int pstride, int maxw,
                                           T* tape, int64_t tape_stride, int64_t tape_off) {
  const int n_in = net.width[l], n_out = net.width[l + 1];
  const int C = net.C, d = net.d;
  const T* __restrict__ Wt = prep + net.wt_off[l];
  const T* __restrict__ b = prep + net.b_off[l];
  const int ngroups = (npts + PP - 1) / PP;
  for (int item = threadIdx.x; item < n_out * ngroups; item += blockDim.x) {
    const int i = item % n_out, g = item / n_out;
    T acc[PP][MAXC];
#pragma unroll
    for (int q = 0; q < PP; ++q)
#pragma unroll
      for (int c = 0; c < MAXC; ++c) acc[q][c] = T(0);
    if (l == 0) {
      for (int j = 0; j < d; ++j) {
        const T wv = Wt[j * n_out + i];
#pragma unroll
        for (int q = 0; q < PP; ++q) {
          const int pt = min(g * PP + q, npts - 1);
          acc[q][0] += wv * (T)X[(row0 + pt) * d + j];
        }
      }
#pragma unroll
      for (int c = 1; c < MAXC; ++c)
        if (c <= d) {
          const T wv = Wt[(c - 1) * n_out + i];
#pragma unroll
          for (int q = 0; q < PP; ++q) acc[q][c] = wv;
        }
    } else {
      for (int j = 0; j < n_in; ++j) {
        const T wv = Wt[j * n_out + i];
#pragma unroll
        for (int q = 0; q < PP; ++q) {
          const T* xin = in + (g * PP + q) * pstride + j;
#pragma unroll
          for (int c = 0; c < MAXC; ++c)
            if (c < C) acc[q][c] += wv * xin[c * maxw];
        }
      }
    }
    const T bi = b[i];
#pragma unroll
    for (int q = 0; q < PP; ++q) {
      const int pt = g * PP + q;
      if (pt >= npts) continue;
      const T a = acc[q][0] + bi;
      const T t = tanh_t<T>(a);
      const T s1 = T(1) - t * t;
      const T s2 = T(-2) * t * s1;
      T qs = T(0), la = T(0);
#pragma unroll
      for (int c = 1; c < MAXC; ++c) {
        if (c <= d && is_spatial(net, c - 1)) qs += acc[q][c] * acc[q][c];
        if (c == d + 1) la = acc[q][c];
      }
      T* xo = out + pt * pstride + i;
      xo[0] = t;
#pragma unroll
      for (int c = 1; c < MAXC; ++c)
        if (c <= d) xo[c * maxw] = s1 * acc[q][c];
      xo[(d + 1) * maxw] = s1 * la + s2 * qs;
      if (tape) {
        T* tp = tape + pt * tape_stride + tape_off + i;
        tp[0] = t;
#pragma unroll
        for (int c = 1; c < MAXC; ++c)
          if (c <= d) tp[c * n_out] = acc[q][c];
        tp[(d + 1) * n_out] = la;
      }
    }
  }
}

// Output layer (n_out = 1): one warp per point; writes the C output channels to outc[pt*C + c].
template <typename T, int MAXC>
__device__ __forceinline__ void fwd_output(const NetDesc& net, const T* __restrict__ prep, const T* in,
                                           int pstride, int maxw, int npts, T* outc) {
  const int l = net.n_layers - 1;
  const int n_in = net.width[l], C = net.C;
  const T* __restrict__ Wt = prep + net.wt_off[l];
  const T bo = prep[net.b_off[l]];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int pt = warp; pt < npts; pt += nw) {
    T acc[MAXC];
#pragma unroll
    for (int c = 0; c < MAXC; ++c) acc[c] = T(0);
    for (int j = lane; j < n_in; j += 32) {
      const T wv = Wt[j];
      const T* xin = in + pt * pstride + j;
#pragma unroll
      for (int c = 0; c < MAXC; ++c)
        if (c < C) acc[c] += wv * xin[c * maxw];
    }
#pragma unroll
    for (int c = 0; c < MAXC; ++c) acc[c] = warp_sum(acc[c]);
    if (lane == 0) {
#pragma unroll
      for (int c = 0; c < MAXC; ++c)
        if (c < C) outc[pt * C + c] = acc[c] + (c == 0 ? bo : T(0));
    }
  }
}

// Residual of each point from its output channels, and this block's share of the loss.
template <typename T>
__device__ __forceinline__ void residual_and_loss(const NetDesc& net, const PointSet& ps, int64_t row0, int npts,
                                                  const T* outc, double* r_out, double* loss_part,
                                                  double* red /* smem, >= 32 doubles */) {
  const int C = net.C, d = net.d;
  double acc = 0.0;
  for (int pt = threadIdx.x; pt < npts; pt += blockDim.x) {
    const int64_t row = row0 + pt;
    const double u = (double)outc[pt * C], g0 = (double)outc[pt * C + 1], lap = (double)outc[pt * C + d + 1];
    double r;
    if (row < ps.n_int) {
      r = (net.pde == NGD_PDE_HEAT) ? g0 - net.kappa * lap - ps.target[row] : lap + ps.target[row];
    } else {
      r = u - ps.target[row];
    }
    if (r_out) r_out[row] = r;
    acc += ps.w[row] * r * r;
  }
  acc = warp_sum(acc);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0 && loss_part) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    loss_part[blockIdx.x] = s;
  }
}

// ---------------------------------------------------------------------------- residual kernel
template <typename T, int MAXC, int PP>
__global__ void __launch_bounds__(kThreads) k_forward(NetDesc net, PointSet ps, const T* __restrict__ prep,
                                                       int64_t row0, int64_t nrows, int TP, double* r_out,
                                                       double* loss_part, T* tape_g, double* chan_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int C = net.C, maxw = net.max_width;
  const int pstride = C * maxw;
  const int64_t trow0 = row0 + (int64_t)blockIdx.x * TP;
  const int npts = (int)min((int64_t)TP, row0 + nrows - trow0);
  T* bufA = sm;
  T* bufB = sm + (size_t)TP * pstride;
  T* outc = sm + (size_t)2 * TP * pstride;
  T* tape = tape_g ? tape_g + trow0 * net.tape_per_point : nullptr;
  int64_t toff = 0;
  for (int l = 0; l < net.n_layers - 1; ++l) {
    fwd_hidden<T, MAXC, PP>(net, l, prep, ps.X, trow0, npts, bufA, bufB, pstride, maxw, tape, net.tape_per_point,
                            toff);
    toff += (int64_t)C * net.width[l + 1];
    __syncthreads();
    T* tmp = bufA; bufA = bufB; bufB = tmp;
  }
  fwd_output<T, MAXC>(net, prep, bufA, pstride, maxw, npts, outc);
  __syncthreads();
  if (chan_out) {                        // u, grad u, Delta u of each point, as float64
    for (int e = threadIdx.x; e < npts * C; e += blockDim.x) chan_out[trow0 * C + e] = (double)outc[e];
  }
  residual_and_loss<T>(net, ps, trow0, npts, outc, r_out, loss_part, red);
}

// ---------------------------------------------------------------------------- Jacobian kernel
// Shared memory per point: tape (C * sum hidden widths) + three [C][maxw] buffers; plus TP*C outputs.
template <typename T, int MAXC, int PP, bool FROM_TAPE>
__global__ void __launch_bounds__(kThreads) k_jacobian(NetDesc net, PointSet ps, const T* __restrict__ prep,
                                                        int64_t row0, int64_t nrows, int TP, T* __restrict__ J,
                                                        int64_t ldJ, double* r_out, double* loss_part,
                                                        const T* __restrict__ tape_g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int C = net.C, d = net.d, maxw = net.max_width;
  const int pstride = C * maxw;
  const int64_t tpp = net.tape_per_point;
  const int64_t trow0 = row0 + (int64_t)blockIdx.x * TP;
  const int npts = (int)min((int64_t)TP, row0 + nrows - trow0);
  T* tape = sm;
  T* bufA = sm + (size_t)TP * tpp;
  T* bufB = bufA + (size_t)TP * pstride;
  T* bufX = bufB + (size_t)TP * pstride;
  T* outc = bufX + (size_t)TP * pstride;

  if (FROM_TAPE) {
    const int64_t n = (int64_t)npts * tpp;
    const T* src = tape_g + trow0 * tpp;
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) tape[k] = src[k];
    __syncthreads();
  } else {
    // Forward: hidden layers ping-pong between bufA and bufB and fill the smem tape.
    T* in = bufA;
    T* out = bufB;
    int64_t toff = 0;
    for (int l = 0; l < net.n_layers - 1; ++l) {
      fwd_hidden<T, MAXC, PP>(net, l, prep, ps.X, trow0, npts, in, out, pstride, maxw, tape, tpp, toff);
      toff += (int64_t)C * net.width[l + 1];
      __syncthreads();
      T* tmp = in; in = out; out = tmp;
    }
    fwd_output<T, MAXC>(net, prep, in, pstride, maxw, npts, outc);
    __syncthreads();
    if (r_out || loss_part) residual_and_loss<T>(net, ps, trow0, npts, outc, r_out, loss_part, red);
    __syncthreads();
  }

  // Reverse pass.  bufA holds abar (adjoint of the pre-activation a_l), bufX the layer
  // input X_{l-1}, bufB the adjoint of that input.  Output seeds: the coefficients of r
  // in (u, grad u, Delta u).
  for (int pt = threadIdx.x; pt < npts; pt += blockDim.x) {
    T* A = bufA + pt * pstride;
    for (int c = 0; c < C; ++c) A[c * maxw] = T(0);
    if (trow0 + pt < ps.n_int) {
      if (net.pde == NGD_PDE_HEAT) {
        A[1 * maxw] = T(1);
        A[(d + 1) * maxw] = (T)(-net.kappa);
      } else {
        A[(d + 1) * maxw] = T(1);
      }
    } else {
      A[0] = T(1);
    }
  }
  __syncthreads();

  // tape offsets of the hidden layers
  int64_t toffs[kMaxLayers];
  {
    int64_t o = 0;
    for (int l = 0; l < net.n_layers - 1; ++l) {
      toffs[l] = o;
      o += (int64_t)C * net.width[l + 1];
    }
  }

  for (int l = net.n_layers - 1; l >= 0; --l) {
    const int n_in = net.width[l], n_out = net.width[l + 1];
    if (l >= 1) {
      // X_{l-1} from the tape of hidden layer l-1 (width n_in).
      const int64_t to = toffs[l - 1];
      for (int item = threadIdx.x; item < npts * n_in; item += blockDim.x) {
        const int pt = item / n_in, j = item - pt * n_in;
        const T* tp = tape + pt * tpp + to + j;
        const T t = tp[0];
        const T s1 = T(1) - t * t, s2 = T(-2) * t * s1;
        T* xo = bufX + pt * pstride + j;
        T qs = T(0);
        for (int k = 0; k < d; ++k) {
          const T ga = tp[(1 + k) * n_in];
          if (is_spatial(net, k)) qs += ga * ga;
          xo[(1 + k) * maxw] = s1 * ga;
        }
        xo[0] = t;
        xo[(d + 1) * maxw] = s1 * tp[(d + 1) * n_in] + s2 * qs;
      }
      __syncthreads();
    }
    // Jacobian entries of W_l (row-major n_out x n_in) and b_l for every point of the tile.
    const int nW = n_out * n_in;
    for (int pt = 0; pt < npts; ++pt) {
      T* __restrict__ Jrow = J + (trow0 - row0 + pt) * ldJ + net.theta_off[l];
      const T* A = bufA + pt * pstride;
      if (l >= 1) {
        const T* Xp = bufX + pt * pstride;
        for (int idx = threadIdx.x; idx < nW; idx += blockDim.x) {
          const int i = idx / n_in, j = idx - i * n_in;
          T v = T(0);
          for (int c = 0; c < C; ++c) v += A[c * maxw + i] * Xp[c * maxw + j];
          Jrow[idx] = v;
        }
      } else {
        const double* xr = ps.X + (trow0 + pt) * d;
        for (int idx = threadIdx.x; idx < nW; idx += blockDim.x) {
          const int i = idx / n_in, j = idx - i * n_in;
          Jrow[idx] = A[i] * (T)xr[j] + A[(1 + j) * maxw + i];
        }
      }
      for (int i = threadIdx.x; i < n_out; i += blockDim.x) Jrow[nW + i] = A[i];
    }
    if (l == 0) break;
    // Adjoint of the layer input: xbar = W_l^T abar, every channel.
    {
      const T* __restrict__ Wr = prep + net.wr_off[l];
      const int ngroups = (npts + PP - 1) / PP;
      for (int item = threadIdx.x; item < n_in * ngroups; item += blockDim.x) {
        const int j = item % n_in, g = item / n_in;
        T acc[PP][MAXC];
#pragma unroll
        for (int q = 0; q < PP; ++q)
#pragma unroll
          for (int c = 0; c < MAXC; ++c) acc[q][c] = T(0);
        for (int i = 0; i < n_out; ++i) {
          const T wv = Wr[i * n_in + j];
#pragma unroll
          for (int q = 0; q < PP; ++q) {
            const T* a = bufA + (g * PP + q) * pstride + i;
#pragma unroll
            for (int c = 0; c < MAXC; ++c)
              if (c < C) acc[q][c] += wv * a[c * maxw];
          }
        }
#pragma unroll
        for (int q = 0; q < PP; ++q) {
          const int pt = g * PP + q;
          if (pt >= npts) continue;
          T* xb = bufB + pt * pstride + j;
#pragma unroll
          for (int c = 0; c < MAXC; ++c)
            if (c < C) xb[c * maxw] = acc[q][c];
        }
      }
    }
    __syncthreads();
    // Adjoint through tanh of hidden layer l-1 (transpose of the Taylor-mode forward):
    //   abar      = s1 xbar + s2 sum_k grad_k a grad_k xbar + (s2 Delta a + s3 q) Delta xbar
    //   grad_k abar = s1 grad_k xbar + 2 s2 grad_k a Delta xbar   (k spatial)
    //   Delta abar  = s1 Delta xbar
    {
      const int64_t to = toffs[l - 1];
      const int nh = n_in;
      for (int item = threadIdx.x; item < npts * nh; item += blockDim.x) {
        const int pt = item / nh, j = item - pt * nh;
        const T* tp = tape + pt * tpp + to + j;
        const T t = tp[0];
        const T s1 = T(1) - t * t, s2 = T(-2) * t * s1, s3 = T(-2) * s1 * (T(1) - T(3) * t * t);
        const T la = tp[(d + 1) * nh];
        const T* xb = bufB + pt * pstride + j;
        const T xbl = xb[(d + 1) * maxw];
        T qs = T(0), sg = T(0);
        for (int k = 0; k < d; ++k) {
          const T ga = tp[(1 + k) * nh];
          if (is_spatial(net, k)) qs += ga * ga;
          sg += ga * xb[(1 + k) * maxw];
        }
        T* A = bufA + pt * pstride + j;
        A[0] = s1 * xb[0] + s2 * sg + (s2 * la + s3 * qs) * xbl;
        for (int k = 0; k < d; ++k) {
          const T ga = tp[(1 + k) * nh];
          A[(1 + k) * maxw] = s1 * xb[(1 + k) * maxw] + (is_spatial(net, k) ? T(2) * s2 * ga * xbl : T(0));
        }
        A[(d + 1) * maxw] = s1 * xbl;
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------- JVP kernel
template <typename T, int MAXC, int PP>
__global__ void __launch_bounds__(kThreads) k_jvp(NetDesc net, PointSet ps, const T* __restrict__ prep,
                                                   const T* __restrict__ prept, int TP, double* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int C = net.C, d = net.d, maxw = net.max_width;
  const int pstride = C * maxw;
  const int64_t trow0 = (int64_t)blockIdx.x * TP;
  const int npts = (int)min((int64_t)TP, ps.N - trow0);
  T* xin = sm;
  T* xdin = xin + (size_t)TP * pstride;
  T* xout = xdin + (size_t)TP * pstride;
  T* xdout = xout + (size_t)TP * pstride;
  for (int l = 0; l < net.n_layers - 1; ++l) {
    const int n_in = net.width[l], n_out = net.width[l + 1];
    const T* __restrict__ Wt = prep + net.wt_off[l];
    const T* __restrict__ Wtd = prept + net.wt_off[l];
    const int ngroups = (npts + PP - 1) / PP;
    for (int item = threadIdx.x; item < n_out * ngroups; item += blockDim.x) {
      const int i = item % n_out, g = item / n_out;
      T acc[PP][MAXC], accd[PP][MAXC];
#pragma unroll
      for (int q = 0; q < PP; ++q)
#pragma unroll
        for (int c = 0; c < MAXC; ++c) acc[q][c] = accd[q][c] = T(0);
      if (l == 0) {
        for (int j = 0; j < d; ++j) {
          const T wv = Wt[j * n_out + i], wdv = Wtd[j * n_out + i];
#pragma unroll
          for (int q = 0; q < PP; ++q) {
            const int pt = min(g * PP + q, npts - 1);
            const T xj = (T)ps.X[(trow0 + pt) * d + j];
            acc[q][0] += wv * xj;
            accd[q][0] += wdv * xj;
          }
        }
#pragma unroll
        for (int c = 1; c < MAXC; ++c)
          if (c <= d) {
            const T wv = Wt[(c - 1) * n_out + i], wdv = Wtd[(c - 1) * n_out + i];
#pragma unroll
            for (int q = 0; q < PP; ++q) {
              acc[q][c] = wv;
              accd[q][c] = wdv;
            }
          }
      } else {
        for (int j = 0; j < n_in; ++j) {
          const T wv = Wt[j * n_out + i], wdv = Wtd[j * n_out + i];
#pragma unroll
          for (int q = 0; q < PP; ++q) {
            const T* x = xin + (g * PP + q) * pstride + j;
            const T* xd = xdin + (g * PP + q) * pstride + j;
#pragma unroll
            for (int c = 0; c < MAXC; ++c)
              if (c < C) {
                const T xv = x[c * maxw];
                acc[q][c] += wv * xv;
                accd[q][c] += wdv * xv + wv * xd[c * maxw];
              }
          }
        }
      }
      const T bi = prep[net.b_off[l] + i], bdi = prept[net.b_off[l] + i];
#pragma unroll
      for (int q = 0; q < PP; ++q) {
        const int pt = g * PP + q;
        if (pt >= npts) continue;
        const T a = acc[q][0] + bi, ad = accd[q][0] + bdi;
        const T t = tanh_t<T>(a);
        const T s1 = T(1) - t * t, s2 = T(-2) * t * s1, s3 = T(-2) * s1 * (T(1) - T(3) * t * t);
        T qs = T(0), qsd = T(0), la = T(0), lad = T(0);
#pragma unroll
        for (int c = 1; c < MAXC; ++c) {
          if (c <= d && is_spatial(net, c - 1)) {
            qs += acc[q][c] * acc[q][c];
            qsd += T(2) * acc[q][c] * accd[q][c];
          }
          if (c == d + 1) {
            la = acc[q][c];
            lad = accd[q][c];
          }
        }
        T* xo = xout + pt * pstride + i;
        T* xdo = xdout + pt * pstride + i;
        xo[0] = t;
        xdo[0] = s1 * ad;
#pragma unroll
        for (int c = 1; c < MAXC; ++c)
          if (c <= d) {
            xo[c * maxw] = s1 * acc[q][c];
            xdo[c * maxw] = s2 * ad * acc[q][c] + s1 * accd[q][c];
          }
        xo[(d + 1) * maxw] = s1 * la + s2 * qs;
        xdo[(d + 1) * maxw] = s1 * lad + s2 * ad * la + s2 * qsd + s3 * ad * qs;
      }
    }
    __syncthreads();
    T* tmp = xin; xin = xout; xout = tmp;
    tmp = xdin; xdin = xdout; xdout = tmp;
  }
  // Output layer: tangent channels only.
  {
    const int l = net.n_layers - 1;
    const int n_in = net.width[l];
    const T* __restrict__ Wt = prep + net.wt_off[l];
    const T* __restrict__ Wtd = prept + net.wt_off[l];
    const T bd = prept[net.b_off[l]];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int pt = warp; pt < npts; pt += nw) {
      T accd[MAXC];
#pragma unroll
      for (int c = 0; c < MAXC; ++c) accd[c] = T(0);
      for (int j = lane; j < n_in; j += 32) {
        const T wv = Wt[j], wdv = Wtd[j];
        const T* x = xin + pt * pstride + j;
        const T* xd = xdin + pt * pstride + j;
#pragma unroll
        for (int c = 0; c < MAXC; ++c)
          if (c < C) accd[c] += wdv * x[c * maxw] + wv * xd[c * maxw];
      }
      T ud = T(0), g0d = T(0), lad = T(0);
#pragma unroll
      for (int c = 0; c < MAXC; ++c) {
        const T s = warp_sum(accd[c]);
        if (c == 0) ud = s + bd;
        if (c == 1) g0d = s;
        if (c == d + 1) lad = s;
      }
      if (lane == 0) {
        const int64_t row = trow0 + pt;
        double v;
        if (row < ps.n_int)
          v = (net.pde == NGD_PDE_HEAT) ? (double)g0d - net.kappa * (double)lad : (double)lad;
        else
          v = (double)ud;
        out[row] = v;
      }
    }
  }
}

// ---------------------------------------------------------------------------- launchers
size_t fwd_smem_per_point(const NetDesc& net, size_t elt) {
  return elt * (2 * (size_t)net.C * net.max_width + net.C);
}
size_t jac_smem_per_point(const NetDesc& net, size_t elt) {
  return elt * ((size_t)net.tape_per_point + 3 * (size_t)net.C * net.max_width + net.C);
}
size_t jvp_smem_per_point(const NetDesc& net, size_t elt) {
  return elt * (4 * (size_t)net.C * net.max_width);
}

static constexpr size_t kSmemBudget = 200 * 1024;

template <int MAXC> constexpr int fwd_pp() { return MAXC <= 8 ? 4 : 2; }
template <int MAXC> constexpr int jvp_pp() { return MAXC <= 8 ? 2 : 1; }

// Largest tile (<= 16 points, a multiple of pp) whose shared memory fits the budget; 0 if none.
static int pick_tp(size_t per_point, int pp, int tp_req) {
  int tp = (int)std::min<size_t>(16, kSmemBudget / per_point);
  if (tp_req > 0) tp = std::min(tp, tp_req);
  tp -= tp % pp;
  return tp;
}

template <typename Kern>
static void set_smem(Kern k, size_t bytes) {
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T, int MAXC>
static int fwd_dispatch(const NetDesc& net, const PointSet& ps, const T* prep, int64_t row0, int64_t nrows,
                        double* r, double* loss_part, T* tape, int tp_req, cudaStream_t s, double* chan) {
  constexpr int PP = fwd_pp<MAXC>();
  const size_t ppb = fwd_smem_per_point(net, sizeof(T));
  const int tp = pick_tp(ppb, PP, tp_req);
  if (tp <= 0) return 0;
  const size_t smem = ppb * tp;
  auto k = k_forward<T, MAXC, PP>;
  set_smem(k, smem);
  const int blocks = (int)((nrows + tp - 1) / tp);
  k<<<blocks, kThreads, smem, s>>>(net, ps, prep, row0, nrows, tp, r, loss_part, tape, chan); note_launch();
  return blocks;
}

template <typename T>
int launch_forward(const NetDesc& net, const PointSet& ps, const T* prep, int64_t row0, int64_t nrows, double* r,
                   double* loss_part, T* tape, int tp, cudaStream_t s, double* chan) {
  if (nrows <= 0) return 0;
  if (net.C <= 4) return fwd_dispatch<T, 4>(net, ps, prep, row0, nrows, r, loss_part, tape, tp, s, chan);
  if (net.C <= 8) return fwd_dispatch<T, 8>(net, ps, prep, row0, nrows, r, loss_part, tape, tp, s, chan);
  if (net.C <= 12) return fwd_dispatch<T, 12>(net, ps, prep, row0, nrows, r, loss_part, tape, tp, s, chan);
  return fwd_dispatch<T, 18>(net, ps, prep, row0, nrows, r, loss_part, tape, tp, s, chan);
}
template int launch_forward<float>(const NetDesc&, const PointSet&, const float*, int64_t, int64_t, double*, double*,
                                   float*, int, cudaStream_t, double*);
template int launch_forward<double>(const NetDesc&, const PointSet&, const double*, int64_t, int64_t, double*,
                                    double*, double*, int, cudaStream_t, double*);

template <typename T, int MAXC>
static int jac_dispatch(const NetDesc& net, const PointSet& ps, const T* prep, int64_t row0, int64_t nrows, T* J,
                        int64_t ldJ, double* r, double* loss_part, const T* tape_in, int tp_req, cudaStream_t s) {
  constexpr int PP = fwd_pp<MAXC>();
  const size_t ppb = jac_smem_per_point(net, sizeof(T));
  const int tp = pick_tp(ppb, PP, tp_req);
  if (tp <= 0) return 0;
  const size_t smem = ppb * tp;
  const int blocks = (int)((nrows + tp - 1) / tp);
  if (tape_in) {
    auto k = k_jacobian<T, MAXC, PP, true>;
    set_smem(k, smem);
    k<<<blocks, kThreads, smem, s>>>(net, ps, prep, row0, nrows, tp, J, ldJ, nullptr, nullptr, tape_in); note_launch();
  } else {
    auto k = k_jacobian<T, MAXC, PP, false>;
    set_smem(k, smem);
    k<<<blocks, kThreads, smem, s>>>(net, ps, prep, row0, nrows, tp, J, ldJ, r, loss_part, nullptr); note_launch();
  }
  return blocks;
}

template <typename T>
int launch_jacobian(const NetDesc& net, const PointSet& ps, const T* prep, int64_t row0, int64_t nrows, T* J,
                    int64_t ldJ, double* r, double* loss_part, const T* tape_in, int tp, cudaStream_t s) {
  if (nrows <= 0) return 0;
  if (net.C <= 4) return jac_dispatch<T, 4>(net, ps, prep, row0, nrows, J, ldJ, r, loss_part, tape_in, tp, s);
  if (net.C <= 8) return jac_dispatch<T, 8>(net, ps, prep, row0, nrows, J, ldJ, r, loss_part, tape_in, tp, s);
  if (net.C <= 12) return jac_dispatch<T, 12>(net, ps, prep, row0, nrows, J, ldJ, r, loss_part, tape_in, tp, s);
  return jac_dispatch<T, 18>(net, ps, prep, row0, nrows, J, ldJ, r, loss_part, tape_in, tp, s);
}
template int launch_jacobian<float>(const NetDesc&, const PointSet&, const float*, int64_t, int64_t, float*, int64_t,
                                    double*, double*, const float*, int, cudaStream_t);
template int launch_jacobian<double>(const NetDesc&, const PointSet&, const double*, int64_t, int64_t, double*,
                                     int64_t, double*, double*, const double*, int, cudaStream_t);

template <typename T, int MAXC>
static int jvp_dispatch(const NetDesc& net, const PointSet& ps, const T* prep, const T* prept, double* out,
                        int tp_req, cudaStream_t s) {
  constexpr int PP = jvp_pp<MAXC>();
  const size_t ppb = jvp_smem_per_point(net, sizeof(T));
  const int tp = pick_tp(ppb, PP, tp_req);
  if (tp <= 0) return 0;
  const size_t smem = ppb * tp;
  auto k = k_jvp<T, MAXC, PP>;
  set_smem(k, smem);
  const int blocks = (int)((ps.N + tp - 1) / tp);
  k<<<blocks, kThreads, smem, s>>>(net, ps, prep, prept, tp, out); note_launch();
  return blocks;
}

template <typename T>
int launch_jvp(const NetDesc& net, const PointSet& ps, const T* prep, const T* prept, double* out, int tp,
               cudaStream_t s) {
  if (net.C <= 4) return jvp_dispatch<T, 4>(net, ps, prep, prept, out, tp, s);
  if (net.C <= 8) return jvp_dispatch<T, 8>(net, ps, prep, prept, out, tp, s);
  if (net.C <= 12) return jvp_dispatch<T, 12>(net, ps, prep, prept, out, tp, s);
  return jvp_dispatch<T, 18>(net, ps, prep, prept, out, tp, s);
}
template int launch_jvp<float>(const NetDesc&, const PointSet&, const float*, const float*, double*, int,
                               cudaStream_t);
template int launch_jvp<double>(const NetDesc&, const PointSet&, const double*, const double*, double*, int,
                                cudaStream_t);

}  // namespace ngd
