// Whole preconditioned CG (Alg. 3, textbook pCG with x0 = 0) for an FP32 stored Jacobian in one
// cooperative persistent kernel: one block per SM, grid barriers between the dependent phases of
// an iteration instead of kernel launches and host round trips.
//
// Per iteration (G = number of blocks; block b owns a contiguous slice of J's rows, of the
// parameter index j and of the Nystrom index k):
//   A  row pass over J: t_n = J_n . p, s_n = w_n t_n, y_b += s_n J_n for the block's rows; one
//      read of J (cp.async ring, L2 evict-first), double-float arithmetic throughout
//   B  q_j = sum_b y_b[j] + mu p_j on the block's j slice; partial p . q
//   C  alpha = r.z / p.q; x += alpha p, r -= alpha q; partial ||r||^2; partial U^T r
//   D  convergence test on ||r||; w2_k = ((lam_ell + mu) / (lam_k + mu) - 1) (U^T r)_k
//   E  z = r + U w2 (Alg. 4, scaled form); partial r . z
//   F  beta = r.z_new / r.z, p = z + beta p
// The preconditioner's U is held as an FP32 pair (Uh + Ul, ~48 bits) in j-major order (U[j, k]
// at j * ell + k, so a block's j slice is one contiguous run): its apply scales the top
// directions by (lam_ell + mu) / (lam_1 + mu) ~ 1e-7, which FP32 U cannot represent, and FP64
// arithmetic runs ~60x slower than FP32 on GB300.  Grid-wide sums are formed identically in
// every block (same operands, same order), so all blocks take the same branch.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "df.cuh"
#include "linalg.cuh"

namespace cg = cooperative_groups;

namespace ngd {
namespace {

constexpr int kT = 384;            // threads per block (one block per SM, 12 warps)
constexpr int kW = kT / 32;        // warps per block
constexpr int kMaxSlice = 256;     // largest j slice per block (p <= kMaxSlice * G)

__device__ __forceinline__ uint64_t evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src, uint64_t pol) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem_src), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Block-wide sum, the same value in every thread and in every block given the same inputs.
// red: kT + 1 doubles.  Only warp 0 does FP64 arithmetic (the FP64 pipe is narrow on GB300).
__device__ __forceinline__ double block_allsum(double v, double* red) {
  __syncthreads();
  red[threadIdx.x] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    // pairwise tree over the kT / 32 values of each lane: short FP64 dependency chains
    double v8[kT / 32];
#pragma unroll
    for (int i = 0; i < kT / 32; ++i) v8[i] = red[threadIdx.x + 32 * i];
#pragma unroll
    for (int w = 1; w < kT / 32; w *= 2)
#pragma unroll
      for (int i = 0; i + w < kT / 32; i += 2 * w) v8[i] += v8[i + w];
    double s = v8[0];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) red[kT] = s;
  }
  __syncthreads();
  return red[kT];
}

// sum over the G blocks of the solve of red[b * 4 + slot] (G <= kT)
__device__ __forceinline__ double grid_total(const double* red, int slot, double* sred, int G) {
  const double v = (int)threadIdx.x < G ? __ldcg(red + threadIdx.x * 4 + slot) : 0.0;
  return block_allsum(v, sred);
}

// Barrier of the blocks of one solve.  A single-problem launch uses the cooperative grid barrier;
// a multi-problem launch (one block group per problem, all groups co-resident in one cooperative
// launch) uses the group's arrival counter a.bar: block arrivals of one barrier make up one
// generation of gG counts, and a block waits until its generation is complete.  The wait is
// bounded (a.wait_cycles); when it runs out the solve's status gets kStatTimeout, and every later
// barrier of the solve returns at once (the loop then ends at its next convergence test).
__device__ __forceinline__ void gsync(const FusedPcgArgs& a, int gG, cg::grid_group& grid) {
  if (!a.bar) {
    grid.sync();
    return;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile int* st = &a.sc->status;
    if (!(*st & kStatTimeout)) {
      __threadfence();
      const unsigned arrived = atomicAdd(a.bar, 1u) + 1u;
      const unsigned target = (arrived + (unsigned)gG - 1u) / (unsigned)gG * (unsigned)gG;
      const long long t0 = clock64();
      for (;;) {
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a.bar) : "memory");
        if ((int)(v - target) >= 0) break;
        if (clock64() - t0 > a.wait_cycles) {
          atomicOr(&a.sc->status, kStatTimeout);
          break;
        }
      }
    }
  }
  __syncthreads();
}


// The block's slice [c0, c1) of the parameter index j: starts on multiples of 4, so that the
// slice's parts of 4-aligned arrays are read as float4.
__device__ __forceinline__ void col_slice(int64_t p, int b, int G, int64_t& c0, int64_t& c1) {
  const int64_t n4 = (p + 3) / 4;
  c0 = 4 * (n4 * b / G);
  c1 = min(p, 4 * (n4 * (b + 1) / G));
}

constexpr int kMaxKSlice = 16;     // largest k slice per block (ell <= kMaxKSlice * G)

struct Smem {
  double coef[kMaxKSlice];          // (lam_ell + mu) / (lam_k + mu) - 1 for the block's k slice
  DF dpart[6][kT / 64];             // phase A: per ring stage, the dot group's warp sums
  double dred[kT + 1];
  float2 rs[kMaxSlice];               // r on the block's j slice, split (phase C -> U^T r)
  double rd[kMaxSlice];               // r on the block's j slice (phase C -> phase E)
};

// Phase A: y_b = sum over the block's rows n of w_n (J_n . v) J_n, written as an FP32 pair.
// Warp-specialised: the first half of the warps (the dot group) stream the rows into a
// shared-memory ring with cp.async and form s_n = w_n (J_n . v); the second half (the update
// group) adds s_n J_n into the block's partial y.  Both groups cover every 16-byte slot of a row
// (thread g of either group owns slots g + kGT c, c < CG), so the update of row n overlaps the
// dot product and reduction of later rows.  Hand-over through named barriers, per ring stage st:
//   FULL[st]  : the dot group arrives after row n's data landed and its warp sums of J_n . v
//               are in sm.dpart[st]; the update group waits on it and forms s_n;
//   EMPTY[st] : the update group arrives after its last read of row n, if row n + S exists;
//               the dot group waits on it before copying row n + S into the stage.
// Each barrier has at most one generation outstanding, and both groups follow the same row
// count, so arrivals and waits pair up.  Slots past the end of a row are never copied and stay
// zero (cleared here by their owners before the first FULL arrival).  v arrives split
// (a.vhf + a.vlf), both words in the dot group's registers.
constexpr int kGT = kT / 2;         // threads per group
constexpr int kMaxStages = 6;
constexpr int kBarFull = 1, kBarEmpty = 1 + kMaxStages;   // named barriers 1..12

__device__ __forceinline__ void nbar_sync(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void nbar_arrive(int id, int count) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}

template <int CG, int S>
__device__ __forceinline__ void gv_rows(const FusedPcgArgs& a, int gb, int gG, float4* ring, Smem& sm) {
  constexpr int PD = S - 2;                      // rows prefetched ahead of the dot group
  static_assert(S >= 3 && S <= kMaxStages, "ring stages");
  const int tid = threadIdx.x, lane = tid & 31;
  const int g = tid % kGT;
  const bool dot_group = tid < kGT;
  const int G = gG, b = gb;
  const int nv4 = (int)(a.ldJ / 4);
  const int64_t rb0 = a.N * b / G, rb1 = a.N * (b + 1) / G;
  const int nrows = (int)(rb1 - rb0);
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  if (dot_group) {
    const int dw = tid >> 5;                     // warp of the dot group
    f2x vh[CG][2], vl[CG][2];
#pragma unroll
    for (int c = 0; c < CG; ++c) {
      const int s = g + c * kGT;
      const float4 h = s < nv4 ? __ldcg(reinterpret_cast<const float4*>(a.vhf) + s) : zero4;
      const float4 l = s < nv4 ? __ldcg(reinterpret_cast<const float4*>(a.vlf) + s) : zero4;
      vh[c][0] = pk2(h.x, h.y);
      vh[c][1] = pk2(h.z, h.w);
      vl[c][0] = pk2(l.x, l.y);
      vl[c][1] = pk2(l.z, l.w);
      if (s >= nv4) {
#pragma unroll
        for (int st = 0; st < S; ++st) ring[(st * CG + c) * kGT + g] = zero4;
      }
    }
    const uint64_t pol = evict_first_policy();
    auto issue = [&](int k) {                    // row rb0 + k into stage k % S (one commit group)
      if (k < nrows) {
        if (k >= S) nbar_sync(kBarEmpty + k % S, kT);
        const float4* src = reinterpret_cast<const float4*>(a.J + (rb0 + k) * a.ldJ) + g;
        float4* dst = ring + (k % S) * CG * kGT + g;
#pragma unroll
        for (int c = 0; c < CG; ++c)
          if (g + c * kGT < nv4) cp_async16(dst + c * kGT, src + c * kGT, pol);
      }
      cp_async_commit();
    };
#pragma unroll
    for (int i = 0; i < PD; ++i) issue(i);
    for (int k = 0; k < nrows; ++k) {
      issue(k + PD);
      cp_async_wait<PD>();
      const int st = k % S;
      const ulonglong2* row = reinterpret_cast<const ulonglong2*>(ring + st * CG * kGT + g);
      DF2 d0{0ull, 0ull}, d1{0ull, 0ull}, d2{0ull, 0ull}, d3{0ull, 0ull};
#pragma unroll
      for (int c = 0; c < CG; c += 2) {
        const ulonglong2 jv = row[c * kGT];
        df2_add_prod_nj(d0, jv.x, vh[c][0], vl[c][0]);
        df2_add_prod_nj(d1, jv.y, vh[c][1], vl[c][1]);
        if (c + 1 < CG) {
          const ulonglong2 jw = row[(c + 1) * kGT];
          df2_add_prod_nj(d2, jw.x, vh[c + 1][0], vl[c + 1][0]);
          df2_add_prod_nj(d3, jw.y, vh[c + 1][1], vl[c + 1][1]);
        }
      }
      DF q[8];
      df2_split(d0, q[0], q[1]);
      df2_split(d1, q[2], q[3]);
      df2_split(d2, q[4], q[5]);
      df2_split(d3, q[6], q[7]);
      DF t = df_add(df_add(df_add(q[0], q[1]), df_add(q[2], q[3])), df_add(df_add(q[4], q[5]), df_add(q[6], q[7])));
      t = warp_sum_df(t);
      if (lane == 0) sm.dpart[st][dw] = t;
      nbar_arrive(kBarFull + st, kT);
    }
    cp_async_wait<0>();
  } else {
    DF2 ya[CG][2];
#pragma unroll
    for (int c = 0; c < CG; ++c) ya[c][0] = ya[c][1] = DF2{0ull, 0ull};
    for (int k = 0; k < nrows; ++k) {
      const int st = k % S;
      const float wh = __ldg(a.wh + rb0 + k), wl = __ldg(a.wl + rb0 + k);
      nbar_sync(kBarFull + st, kT);
      // every thread of the update group combines the dot group's warp sums itself
      DF s = sm.dpart[st][0];
#pragma unroll
      for (int w = 1; w < kGT / 32; ++w) s = df_add(s, sm.dpart[st][w]);
      const DF sn = df_mul(s, wh, wl);
      const f2x sh = pk2(sn.hi, sn.hi), nsh = pk2(-sn.hi, -sn.hi), sl = pk2(sn.lo, sn.lo);
      const ulonglong2* row = reinterpret_cast<const ulonglong2*>(ring + st * CG * kGT + g);
#pragma unroll
      for (int c = 0; c < CG; ++c) {
        const ulonglong2 jv = row[c * kGT];
        df2_add_prod(ya[c][0], jv.x, sh, nsh, sl);
        df2_add_prod(ya[c][1], jv.y, sh, nsh, sl);
      }
      if (k + S < nrows) nbar_arrive(kBarEmpty + st, kT);
    }
    float4* oh = reinterpret_cast<float4*>(a.yph + (int64_t)b * a.ldJ);
    float4* ol = reinterpret_cast<float4*>(a.ypl + (int64_t)b * a.ldJ);
#pragma unroll
    for (int c = 0; c < CG; ++c) {
      const int s = g + c * kGT;
      if (s < nv4) {
        float h0, h1, h2, h3, l0, l1, l2, l3;
        upk2(ya[c][0].hi, h0, h1);
        upk2(ya[c][1].hi, h2, h3);
        upk2(ya[c][0].lo, l0, l1);
        upk2(ya[c][1].lo, l2, l3);
        __stcg(oh + s, make_float4(h0, h1, h2, h3));
        __stcg(ol + s, make_float4(l0, l1, l2, l3));
      }
    }
  }
}

// The block's j slice of v, split into FP32 pairs for phase A.
__device__ __forceinline__ void split_slice(const FusedPcgArgs& a, int gb, int gG, const double* v) {
  int64_t cb0, cb1;
  col_slice(a.p, gb, gG, cb0, cb1);
  for (int64_t j = cb0 + threadIdx.x; j < cb1; j += kT) {
    float h, l;
    split_df(v[j], h, l);
    __stcg(a.vhf + j, h);
    __stcg(a.vlf + j, l);
  }
}

// Phase B: q_j = sum_b y_b[j] + mu v_j on the block's j slice; returns the block's sum of v_j q_j.
// Thread (c4, g): columns 4 c4 .. 4 c4 + 3 of the slice, partials b = g, g + kW, ...; scr: shared
// scratch of kW x 32 x 4 double-float values.
__device__ __forceinline__ double gv_finish(const FusedPcgArgs& a, int gb, int gG, const double* v, double mu,
                                            double* q, DF* scr) {
  const int tid = threadIdx.x, G = gG;
  int64_t cb0, cb1;
  col_slice(a.p, gb, G, cb0, cb1);
  const int c4 = tid & 31, g = tid >> 5;                 // 32 column quads x kW partial groups
  double vq = 0.0;
  for (int64_t j0 = cb0; j0 < cb1; j0 += 128) {
    const int64_t j = j0 + 4 * c4;
    DF acc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    if (j < cb1) {
#pragma unroll 4
      for (int bb = g; bb < G; bb += kW) {
        const float4 h = __ldcg(reinterpret_cast<const float4*>(a.yph + (int64_t)bb * a.ldJ + j));
        const float4 l = __ldcg(reinterpret_cast<const float4*>(a.ypl + (int64_t)bb * a.ldJ + j));
        acc[0] = df_add(acc[0], DF{h.x, l.x});
        acc[1] = df_add(acc[1], DF{h.y, l.y});
        acc[2] = df_add(acc[2], DF{h.z, l.z});
        acc[3] = df_add(acc[3], DF{h.w, l.w});
      }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) scr[(g * 32 + c4) * 4 + e] = acc[e];
    __syncthreads();
    if (tid < 128) {
      const int cc = tid >> 2, e = tid & 3;              // one thread per column
      const int64_t jc = j0 + tid;
      if (jc < cb1) {
        DF s = scr[cc * 4 + e];
#pragma unroll
        for (int g2 = 1; g2 < kW; ++g2) s = df_add(s, scr[(g2 * 32 + cc) * 4 + e]);
        const double vj = __ldcg(v + jc);
        const double qj = df_to_double(s) + mu * vj;
        q[jc] = qj;
        vq += vj * qj;
      }
    }
    __syncthreads();
  }
  return vq;
}

// The block's j slice of U (rows cb0 .. cb0 + ncol of Uh and Ul, ldu words each, contiguous)
// passes through dynamic shared memory for the preconditioner: after a 16 KB head (the scaled
// U^T r of phase E, or scratch) come two buffers of R rows; chunk i of the slice goes to buffer
// i % 2, chunk 0 holding the remainder rows so that the later chunks are full.  Phase C walks
// the chunks upwards and phase E downwards, so E starts on the two chunks C left resident and
// copies only the others, each while the previous chunk is being used (cp.async groups).  The
// row pass (phase A) reuses the space as its ring, so C always copies the whole slice.
constexpr int kHead = 16 * 1024;

struct UStage {
  float* buf0;                       // buffer b at buf0 + b * bstride: R * ldu high, then R * ldu low words
  int bstride, R, nch, len0;
  __device__ __forceinline__ float* buf(int i) const { return buf0 + (i & 1) * bstride; }
  __device__ __forceinline__ int start(int i) const { return i == 0 ? 0 : len0 + (i - 1) * R; }
  __device__ __forceinline__ int len(int i) const { return i == 0 ? len0 : R; }
};

__device__ __forceinline__ unsigned dyn_smem_bytes() {
  unsigned v;
  asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(v));   // volatile: not hoisted out of the CG loop
  return v;
}

__device__ __forceinline__ UStage ustage(const FusedPcgArgs& a, unsigned char* dsm, int ncol) {
  UStage st;
  const unsigned half = ((dyn_smem_bytes() - kHead) / 2) & ~15u;
  st.buf0 = reinterpret_cast<float*>(dsm + kHead);
  st.bstride = (int)(half / 4);
  st.R = (int)(half / (8u * (unsigned)a.ldu));
  st.nch = ncol > 0 ? (ncol + st.R - 1) / st.R : 0;
  st.len0 = ncol - (st.nch - 1) * st.R;
  return st;
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem_src) : "memory");
}

// Copy chunk i of the slice into its buffer (one commit group).
__device__ __forceinline__ void ustage_issue(const FusedPcgArgs& a, const UStage& st, int64_t cb0, int i) {
  const int n16 = st.len(i) * a.ldu / 4;
  const int64_t off = (cb0 + st.start(i)) * a.ldu;
  float* dh = st.buf(i);
  float* dl = dh + st.R * a.ldu;
  for (int e = threadIdx.x; e < 2 * n16; e += kT) {
    const bool lo = e >= n16;
    const int o = 4 * (lo ? e - n16 : e);
    cp_async16((lo ? dl : dh) + o, (lo ? a.Ul : a.Uh) + off + o);
  }
  cp_async_commit();
}

// Phase C's partial U^T r over the block's j slice (r_j already split into sm.rs), written to
// w1p[b, :].  Thread (grp, t) takes k quads t, t + nthr (U rows padded to ldu, a multiple of 4)
// and rows grp, grp + ngrp, ... of every chunk; the ngrp row groups are combined at the end
// through the head of shared memory.  Leaves the last two chunks in their buffers.
constexpr int kUQ = 2;             // k quads per thread: ell <= kUQ * 4 * kT
__device__ __forceinline__ void utr_partial(const FusedPcgArgs& a, int gb, int64_t cb0, int ncol, Smem& sm,
                                            unsigned char* dsm) {
  const UStage st = ustage(a, dsm, ncol);
  const int nk4 = a.ldu / 4;
  const int ngrp = max(1, min(8, kT / nk4)), nthr = kT / ngrp;
  const int grp = threadIdx.x / nthr, t = threadIdx.x % nthr;
  DF acc[kUQ][4];
#pragma unroll
  for (int q = 0; q < kUQ; ++q)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[q][e] = DF{0.f, 0.f};
  if (st.nch > 0) ustage_issue(a, st, cb0, 0);
  if (st.nch > 1) ustage_issue(a, st, cb0, 1);
  for (int i = 0; i < st.nch; ++i) {
    if (i + 1 < st.nch) cp_async_wait<1>();
    else cp_async_wait<0>();
    __syncthreads();
    const int r0 = st.start(i), nr = st.len(i);
    const float4* bh = reinterpret_cast<const float4*>(st.buf(i));
    const float4* bl = bh + st.R * nk4;
    if (grp < ngrp) {
#pragma unroll 2
      for (int rr = grp; rr < nr; rr += ngrp) {
        const float2 rv = sm.rs[r0 + rr];
#pragma unroll
        for (int q = 0; q < kUQ; ++q) {
          const int k4 = t + q * nthr;
          if (k4 < nk4) {
            const float4 h = bh[rr * nk4 + k4], l = bl[rr * nk4 + k4];
            df_add_prod2(acc[q][0], h.x, l.x, rv.x, rv.y);
            df_add_prod2(acc[q][1], h.y, l.y, rv.x, rv.y);
            df_add_prod2(acc[q][2], h.z, l.z, rv.x, rv.y);
            df_add_prod2(acc[q][3], h.w, l.w, rv.x, rv.y);
          }
        }
      }
    }
    if (i + 2 < st.nch) {
      __syncthreads();
      ustage_issue(a, st, cb0, i + 2);
    }
  }
  DF* scr = reinterpret_cast<DF*>(dsm);             // (ngrp - 1) x nthr x 4 values (ngrp > 1: one quad)
  if (ngrp > 1 && grp >= 1 && grp < ngrp) {
#pragma unroll
    for (int e = 0; e < 4; ++e) scr[((grp - 1) * nthr + t) * 4 + e] = acc[0][e];
  }
  __syncthreads();
  if (grp == 0) {
#pragma unroll
    for (int q = 0; q < kUQ; ++q) {
      const int k4 = t + q * nthr;
      if (k4 < nk4) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int k = 4 * k4 + e;
          DF s = acc[q][e];
          for (int g2 = 1; g2 < ngrp; ++g2) s = df_add(s, scr[((g2 - 1) * nthr + t) * 4 + e]);
          if (k < a.ell) __stcg(a.w1p + (int64_t)gb * a.ell + k, make_float2(s.hi, s.lo));
        }
      }
    }
  }
  __syncthreads();
}

// Phase E: z_j = r_j + sum_k U[j, k] w2[k] on the block's j slice (w2 in the head of shared
// memory), chunks taken downwards starting with the two that phase C left resident; a warp takes
// two rows of a chunk at a time, lanes over k quads.  Returns the thread's part of r . z.
__device__ __forceinline__ double precond_rows(const FusedPcgArgs& a, int64_t cb0, int ncol, Smem& sm,
                                               unsigned char* dsm) {
  const UStage st = ustage(a, dsm, ncol);
  const float2* w2s = reinterpret_cast<const float2*>(dsm);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nk4 = a.ldu / 4;
  double rzp = 0.0;
  for (int i = st.nch - 1; i >= 0; --i) {
    if (i >= 1 && i + 2 <= st.nch) cp_async_wait<1>();   // chunk i - 1 may still be in flight
    else cp_async_wait<0>();
    __syncthreads();
    const int r0 = st.start(i), nr = st.len(i);
    const float4* bh = reinterpret_cast<const float4*>(st.buf(i));
    const float4* bl = bh + st.R * nk4;
    for (int j0 = 2 * warp; j0 < nr; j0 += 2 * kW) {
      const bool two = j0 + 1 < nr;
      const float4* uh0 = bh + j0 * nk4;
      const float4* ul0 = bl + j0 * nk4;
      const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
      DF acc0{0.f, 0.f}, acc1{0.f, 0.f};
#pragma unroll 1
      for (int k4 = lane; k4 < nk4; k4 += 32) {
        const float4 wa = reinterpret_cast<const float4*>(w2s)[2 * k4];       // w2[4 k4], w2[4 k4 + 1]
        const float4 wb = reinterpret_cast<const float4*>(w2s)[2 * k4 + 1];   // w2[4 k4 + 2], w2[4 k4 + 3]
        const float4 h0 = uh0[k4], l0 = ul0[k4];
        const float4 h1 = two ? uh0[nk4 + k4] : zero4, l1 = two ? ul0[nk4 + k4] : zero4;
        df_add_prod2(acc0, h0.x, l0.x, wa.x, wa.y);
        df_add_prod2(acc0, h0.y, l0.y, wa.z, wa.w);
        df_add_prod2(acc0, h0.z, l0.z, wb.x, wb.y);
        df_add_prod2(acc0, h0.w, l0.w, wb.z, wb.w);
        df_add_prod2(acc1, h1.x, l1.x, wa.x, wa.y);
        df_add_prod2(acc1, h1.y, l1.y, wa.z, wa.w);
        df_add_prod2(acc1, h1.z, l1.z, wb.x, wb.y);
        df_add_prod2(acc1, h1.w, l1.w, wb.z, wb.w);
      }
      const DF s = warp_reduce_scatter2(acc0, acc1);     // lanes 0..15: row j0, 16..31: row j0 + 1
      const int q = lane >> 4;
      if ((lane & 15) == 0 && (q == 0 || two)) {
        const int jj = r0 + j0 + q;
        const double rj = sm.rd[jj], zj = rj + df_to_double(s);
        a.z[cb0 + jj] = zj;
        rzp += rj * zj;
      }
    }
    if (i >= 2) {
      __syncthreads();
      ustage_issue(a, st, cb0, i - 2);
    }
  }
  return rzp;
}

template <int CG, int S>
__device__ __forceinline__ void pcg_body(const FusedPcgArgs& a, const int gb, const int gG) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ __align__(16) unsigned char dsm[];
  float4* ring = reinterpret_cast<float4*>(dsm);
  float2* w2s = reinterpret_cast<float2*>(dsm);          // phase E only (aliases the ring)
  DF* scr = reinterpret_cast<DF*>(dsm);                  // phase B only (aliases the ring)
  __shared__ Smem sm;
  const int tid = threadIdx.x, G = gG, b = gb;
  const double mu = a.mu_d ? *a.mu_d : a.mu_h;

  if (a.mode == 1) {                                     // q = (G + mu I) v, v = a.pv
    split_slice(a, gb, gG, a.pv);
    gsync(a, gG, grid);
    gv_rows<CG, S>(a, gb, gG, ring, sm);
    gsync(a, gG, grid);
    gv_finish(a, gb, gG, a.pv, mu, a.q, scr);
    return;
  }

  int64_t cb0, cb1;
  col_slice(a.p, b, G, cb0, cb1);
  const int ncol = (int)(cb1 - cb0);
  const int kb0 = (int)((int64_t)a.ell * b / G), kb1 = (int)((int64_t)a.ell * (b + 1) / G);
  const bool pre = a.ell > 0;
  if (pre && tid < kb1 - kb0) {     // the scaled preconditioner's coefficients, once per solve
    const double lam_l = a.lam[a.ell - 1];
    sm.coef[tid] = (lam_l + mu) / (a.lam[kb0 + tid] + mu) - 1.0;
  }
  PcgScalars* sc = a.sc;
  const double rtol2 = sc->rtol2;
  const int maxit = sc->maxit;

  // x = 0, r = g, ||g||^2, U^T r
  double rr = 0.0;
  for (int jj = tid; jj < ncol; jj += kT) {
    const double gj = a.g[cb0 + jj];
    a.x[cb0 + jj] = 0.0;
    a.r[cb0 + jj] = gj;
    rr += gj * gj;
    float h, l;
    split_df(gj, h, l);
    sm.rs[jj] = make_float2(h, l);
    sm.rd[jj] = gj;
  }
  rr = block_allsum(rr, sm.dred);
  if (tid == 0) __stcg(a.red + b * 4 + 1, rr);
  if (pre) utr_partial(a, gb, cb0, ncol, sm, dsm);
  gsync(a, gG, grid);

  int it = 0, status = 0;
  double gn2 = 0.0, rn2 = 0.0, rz = 0.0, alpha = 0.0, beta = 0.0, pq = 0.0;
  for (;;) {
    // D: convergence test; finish U^T r and scale it
    rn2 = grid_total(a.red, 1, sm.dred, G);
    bool done;
    if (a.bar && (*(volatile int*)&sc->status & kStatTimeout)) break;   // a group barrier gave up
    if (it == 0) {
      gn2 = rn2;
      done = rn2 == 0.0 || maxit <= 0;
    } else {
      done = rn2 <= rtol2 * gn2 || it >= maxit;
    }
    if (!isfinite(rn2)) {
      status |= kStatNonFinite;
      done = true;
    }
    if (done) break;
    if (pre) {
      const int lane = tid & 31, warp = tid >> 5;
      for (int k = kb0 + warp; k < kb1; k += kW) {
        DF acc{0.f, 0.f};
#pragma unroll 4
        for (int bb = lane; bb < G; bb += 32) {
          const float2 t = __ldcg(a.w1p + (int64_t)bb * a.ell + k);
          acc = df_add(acc, DF{t.x, t.y});
        }
        acc = warp_sum_df(acc);
        if (lane == 0) {
          const double w2 = sm.coef[k - kb0] * df_to_double(acc);
          float h, l;
          split_df(w2, h, l);
          __stcg(a.w2 + k, make_float2(h, l));
        }
      }
      gsync(a, gG, grid);
    }
    // E: z = P^{-1} r on the j slice, r . z
    double rzp = 0.0;
    if (pre) {
      for (int k = tid; k < a.ldu; k += kT) w2s[k] = k < a.ell ? __ldcg(a.w2 + k) : make_float2(0.f, 0.f);
      __syncthreads();
      rzp = precond_rows(a, cb0, ncol, sm, dsm);
    } else {
      for (int jj = tid; jj < ncol; jj += kT) {
        const double rj = a.r[cb0 + jj];
        a.z[cb0 + jj] = rj;
        rzp += rj * rj;
      }
    }
    rzp = block_allsum(rzp, sm.dred);
    if (tid == 0) __stcg(a.red + b * 4 + 2, rzp);
    gsync(a, gG, grid);
    // F: beta, new direction
    {
      const double rz_new = grid_total(a.red, 2, sm.dred, G);
      beta = it == 0 ? 0.0 : rz_new / rz;
      for (int jj = tid; jj < ncol; jj += kT) {
        const int64_t j = cb0 + jj;
        const double pj = it == 0 ? a.z[j] : a.z[j] + beta * a.pv[j];
        a.pv[j] = pj;
        float h, l;
        split_df(pj, h, l);
        __stcg(a.vhf + j, h);
        __stcg(a.vlf + j, l);
      }
      rz = rz_new;
    }
    gsync(a, gG, grid);
    // A, B: q = (G + mu I) p, p . q
    gv_rows<CG, S>(a, gb, gG, ring, sm);
    gsync(a, gG, grid);
    {
      double pqp = gv_finish(a, gb, gG, a.pv, mu, a.q, scr);
      pqp = block_allsum(pqp, sm.dred);
      if (tid == 0) __stcg(a.red + b * 4 + 0, pqp);
    }
    gsync(a, gG, grid);
    // C: alpha, x and r, ||r||^2, U^T r
    pq = grid_total(a.red, 0, sm.dred, G);
    if (!(pq > 0.0) || !isfinite(pq)) {
      status |= isfinite(pq) ? kStatBreakdown : kStatNonFinite;
      break;
    }
    alpha = rz / pq;
    rr = 0.0;
    for (int jj = tid; jj < ncol; jj += kT) {
      const int64_t j = cb0 + jj;
      a.x[j] += alpha * a.pv[j];
      const double rj = a.r[j] - alpha * a.q[j];
      a.r[j] = rj;
      rr += rj * rj;
      float h, l;
      split_df(rj, h, l);
      sm.rs[jj] = make_float2(h, l);
      sm.rd[jj] = rj;
    }
    rr = block_allsum(rr, sm.dred);
    if (tid == 0) __stcg(a.red + b * 4 + 1, rr);
    if (pre) utr_partial(a, gb, cb0, ncol, sm, dsm);
    ++it;
    gsync(a, gG, grid);
  }
  if (b == 0 && tid == 0) {
    sc->gn2 = gn2;
    sc->rn2 = rn2;
    sc->rz = rz;
    sc->pq = pq;
    sc->alpha = alpha;
    sc->beta = beta;
    sc->iters = it;
    sc->cur_iter = it;
    sc->status |= status;
    sc->done = 1;
  }
}

template <int CG, int S>
__global__ void __launch_bounds__(kT, 1) k_pcg_fused(const FusedPcgArgs a) {
  pcg_body<CG, S>(a, (int)blockIdx.x, (int)gridDim.x);
}

// Many independent solves in one cooperative launch: problem j owns the blocks
// [tab[j].gb0, tab[j].gb0 + tab[j].gG) (groups in increasing gb0 order) and synchronises them
// with its own barrier counter.
template <int CG, int S>
__global__ void __launch_bounds__(kT, 1) k_pcg_fused_multi(const FusedPcgArgs* __restrict__ tab, int nprob) {
  int j = 0;
  while (j + 1 < nprob && (int)blockIdx.x >= tab[j + 1].gb0) ++j;
  const FusedPcgArgs& a = tab[j];
  pcg_body<CG, S>(a, (int)blockIdx.x - a.gb0, a.gG);
}

constexpr int kMaxCG = 12;       // slots per group thread: p <= 4 * kGT * kMaxCG = 9216
constexpr int kSmemBudget = 210 * 1024;

// ring stages, at most kMaxStages
template <int CG>
constexpr int stages_for() {
  return std::min(kMaxStages, kSmemBudget / (CG * kGT * 16));
}

// Launch of the fused solve with CG slots per group thread: one problem on G blocks (tab null),
// or nprob problems from the device table tab on G blocks in all.
template <int CG>
cudaError_t launch_cg(const FusedPcgArgs& a, int G, cudaStream_t s, const FusedPcgArgs* tab = nullptr,
                      int nprob = 0) {
  constexpr int S = stages_for<CG>();
  static_assert(S >= 3, "shared-memory ring too small");
  auto kern = k_pcg_fused<CG, S>;
  auto kern_multi = k_pcg_fused_multi<CG, S>;
  // dynamic shared memory: the whole budget (one block per SM in any case), shared by the ring of
  // phase A and the head plus the two U buffers of phases C and E (16 KB + 2 rows of U at least)
  constexpr size_t smem = kSmemBudget;
  static_assert((size_t)S * CG * kGT * 16 <= smem && kHead + 2 * 8 * 2048 <= smem, "dynamic shared memory");
  static std::mutex mu;
  static int configured_dev = -1, per_sm = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (configured_dev != dev) {
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      e = cudaFuncSetAttribute(kern_multi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kT, smem);
      if (e != cudaSuccess) return e;
      configured_dev = dev;
    }
  }
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  if (tab) {
    const FusedPcgArgs* t = tab;
    int n = nprob;
    void* params[] = {&t, &n};
    e = cudaLaunchCooperativeKernel((const void*)kern_multi, G, kT, params, smem, s);
  } else {
    FusedPcgArgs args = a;
    void* params[] = {&args};
    e = cudaLaunchCooperativeKernel((const void*)kern, G, kT, params, smem, s);
  }
  note_launch();
  return e;
}

int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  }
  return n;
}

}  // namespace

int fused_pcg_blocks() { return std::min(num_sms(), kT); }

int fused_pcg_slots(int64_t ldJ) { return (int)((ldJ / 4 + kGT - 1) / kGT); }

bool fused_pcg_supported_on(int64_t p, int64_t ldJ, int ell, int G) {
  const int64_t cg = fused_pcg_slots(ldJ);
  return G >= 1 && G <= kT && ldJ % 4 == 0 && cg >= 1 && cg <= kMaxCG &&
         4 * (((p + 3) / 4 + G - 1) / G) <= kMaxSlice && ell >= 0 && ell <= 2048 && ell <= kMaxKSlice * G;
}

bool fused_pcg_supported(int64_t p, int64_t ldJ, int ell) {
  return fused_pcg_supported_on(p, ldJ, ell, fused_pcg_blocks());
}

int fused_pcg_min_blocks(int64_t p, int ell) {
  const int64_t by_p = ((p + 3) / 4 + kMaxSlice / 4 - 1) / (kMaxSlice / 4);
  const int64_t by_ell = (ell + kMaxKSlice - 1) / kMaxKSlice;
  return (int)std::max<int64_t>(1, std::max(by_p, by_ell));
}

static cudaError_t launch_by_slots(const FusedPcgArgs& a, int G, cudaStream_t s, const FusedPcgArgs* tab, int nprob) {
  switch ((fused_pcg_slots(a.ldJ) + 1) / 2) {     // slots per group thread, rounded up to even
    case 1: return launch_cg<2>(a, G, s, tab, nprob);
    case 2: return launch_cg<4>(a, G, s, tab, nprob);
    case 3: return launch_cg<6>(a, G, s, tab, nprob);
    case 4: return launch_cg<8>(a, G, s, tab, nprob);
    case 5: return launch_cg<10>(a, G, s, tab, nprob);
    default: return launch_cg<12>(a, G, s, tab, nprob);
  }
}

cudaError_t launch_pcg_fused(const FusedPcgArgs& a, cudaStream_t s) {
  if (!fused_pcg_supported(a.p, a.ldJ, a.ell)) return cudaErrorInvalidValue;
  return launch_by_slots(a, fused_pcg_blocks(), s, nullptr, 0);
}

cudaError_t launch_pcg_fused_multi(const FusedPcgArgs* tab_dev, const FusedPcgArgs* tab_host, int nprob,
                                   cudaStream_t s) {
  if (nprob < 1) return cudaErrorInvalidValue;
  const int slots = (fused_pcg_slots(tab_host[0].ldJ) + 1) / 2;
  int G = 0;
  for (int j = 0; j < nprob; ++j) {
    const FusedPcgArgs& a = tab_host[j];
    if (a.gb0 != G || (fused_pcg_slots(a.ldJ) + 1) / 2 != slots || !a.bar ||
        !fused_pcg_supported_on(a.p, a.ldJ, a.ell, a.gG))
      return cudaErrorInvalidValue;
    G += a.gG;
  }
  if (G > fused_pcg_blocks()) return cudaErrorInvalidValue;
  return launch_by_slots(tab_host[0], G, s, tab_dev, nprob);
}

// U (column-major, leading dimension ldu, p x ell, float or double) -> Uh + Ul in j-major order
// with rows padded to ldr = ell rounded up to a multiple of 4 (U[j, k] at j * ldr + k, zero for
// k >= ell); 32 x 32 tiles transposed through shared memory.
template <typename TU>
__global__ void k_split_transpose_df(const TU* __restrict__ U, int64_t ldu, int64_t p, int ell, float* __restrict__ Uh,
                                     float* __restrict__ Ul) {
  __shared__ float th[32][33], tl[32][33];
  const int64_t j0 = (int64_t)blockIdx.x * 32;
  const int k0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int i = ty; i < 32; i += 8) {
    const int64_t j = j0 + tx;
    const int k = k0 + i;
    float h = 0.f, l = 0.f;
    if (j < p && k < ell) split_df((double)U[j + (int64_t)k * ldu], h, l);
    th[i][tx] = h;
    tl[i][tx] = l;
  }
  __syncthreads();
  const int ldr = (ell + 3) / 4 * 4;
  for (int i = ty; i < 32; i += 8) {
    const int64_t j = j0 + i;
    const int k = k0 + tx;
    if (j < p && k < ldr) {
      Uh[j * ldr + k] = th[tx][i];   // zero for k >= ell (tile loaded as zero there)
      Ul[j * ldr + k] = tl[tx][i];
    }
  }
}
template <typename TU>
void launch_split_transpose_df(const TU* U, int64_t ldu, int64_t p, int ell, float* Uh, float* Ul, cudaStream_t s) {
  dim3 grid((unsigned)((p + 31) / 32), (unsigned)((ell + 3) / 4 * 4 + 31) / 32);
  k_split_transpose_df<TU><<<grid, 256, 0, s>>>(U, ldu, p, ell, Uh, Ul); note_launch();
}
template void launch_split_transpose_df<float>(const float*, int64_t, int64_t, int, float*, float*, cudaStream_t);
template void launch_split_transpose_df<double>(const double*, int64_t, int64_t, int, float*, float*, cudaStream_t);

}  // namespace ngd
