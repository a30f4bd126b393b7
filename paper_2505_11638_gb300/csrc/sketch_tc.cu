// Nystrom sketch Y = J^T diag(w) (J Omega) on the 5th-generation tensor cores (App. A,
// third step: the only dense contraction of the hot path).
//
// Two GEMMs D = A B^T with both operands K-major:
//   GEMM1  A = J (N x p), B = Omega^T (ell x p)   -> Z = J Omega, epilogue scales row n by w_n
//          and stores Z^T (ell x N), the K-major operand of GEMM2;
//   GEMM2  A = J^T (p x N), B = Z^T (ell x N)     -> Y (p x ell, column-major).
// J^T is a transposed copy made once per linearization.  Operands are TF32 (FP32 bits
// read by the tensor core) or BF16 (rounded to nearest); accumulation is FP32 in TMEM.
//
// Kernel: one 128 x 128 output tile per CTA, six-stage TMA -> shared memory pipeline
// (128-byte swizzle), one elected thread issues tcgen05.mma (kind::tf32 / kind::f16,
// cta_group::1, M = 128, N = 128) into a 128-column TMEM accumulator, four epilogue warps
// drain it with tcgen05.ld.  Every mbarrier wait is bounded (tc_common.cuh: a role whose wait
// runs out stops issuing work, the CTA drains the loads and MMAs already issued, stores
// nothing, records kStatTimeout, frees its TMEM and returns).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "ngd_internal.cuh"
#include "sketch_tc.cuh"
#include "tc_common.cuh"

namespace ngd {

namespace tc {

EncodeFn tensor_map_encoder() {
  static EncodeFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeFn>(p);
  }
  return fn;
}

bool make_tile_map(CUtensorMap* m, const void* base, int elem_bytes, int64_t rows, int64_t cols, int64_t ld,
                   int64_t planes, int64_t plane_ld, int box_rows) {
  EncodeFn enc = tensor_map_encoder();
  if (!enc || (elem_bytes != 2 && elem_bytes != 4) || box_rows < 8 || box_rows > 256) return false;
  const size_t es = (size_t)elem_bytes;
  if ((reinterpret_cast<uintptr_t>(base) & 15) || ((ld * es) & 15) || (planes > 1 && ((plane_ld * es) & 15)))
    return false;
  const CUtensorMapDataType dt = es == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)(ld * es), (cuuint64_t)(plane_ld * es)};
  cuuint32_t box[3] = {(cuuint32_t)(128 / es), (cuuint32_t)box_rows, 1u};
  cuuint32_t estr[3] = {1u, 1u, 1u};
  const cuuint32_t rank = planes > 1 ? 3 : 2;
  const CUresult r = enc(m, dt, rank, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace tc

namespace {

using namespace tc;

constexpr int BM = 128, BN = 128, STAGES = 6;
constexpr int TILE_BYTES = 128 * 128;                    // 128 rows x 128 bytes
constexpr int SMEM_BYTES = 2 * STAGES * TILE_BYTES + 1024 + 256;

struct Epi {
  int mode;            // 0: Z^T with row weights, 1: column-major Y, 2: generic strides
  int out_bf16;        // mode 0: Z^T stored as BF16
  const double* w;     // mode 0 row weights
  void* out;
  int64_t ld_out;      // mode 0: row length of Z^T; mode 1: ld of Y
  int64_t M, Nn;       // valid rows / columns of D
  int64_t ldd_m, ldd_n;
};

template <bool BF16>
__global__ void __launch_bounds__(192, 1) k_tc_gemm(const __grid_constant__ CUtensorMap tmA,
                                                   const __grid_constant__ CUtensorMap tmB, int num_kt, Epi ep,
                                                   int* status, long long wait_cycles) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * TILE_BYTES;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + 2 * STAGES * TILE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* accum = empty + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accum, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tmem_slot, 128);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  int err = 0;   // bit 0: a wait ran out; bit 1: a drain wait ran out too

  if (warp == 0 && lane == 0) {
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    constexpr int BK = BF16 ? 64 : 32;
    int issued = 0;
    for (int kt = 0; kt < num_kt; ++kt) {
      const int s = kt % STAGES;
      if (*abort_flag) break;
      if (kt >= STAGES && !mbar_wait(&empty[s], ((kt / STAGES) - 1) & 1, wait_cycles)) {
        err |= 1;
        *abort_flag = 1;
        break;
      }
      mbar_expect_tx(&full[s], 2 * TILE_BYTES);
      tma_load_2d(sA + s * TILE_BYTES, &tmA, kt * BK, m0, &full[s]);
      tma_load_2d(sB + s * TILE_BYTES, &tmB, kt * BK, n0, &full[s]);
      issued = kt + 1;
    }
    // every load still unconsumed must land before the CTA may exit
    for (int j = issued > STAGES ? issued - STAGES : 0; j < issued; ++j)
      if (!mbar_wait(&full[j % STAGES], (j / STAGES) & 1, kDrainCycles)) err |= 2;
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = make_idesc(BF16 ? 1u : 2u, BM, BN);
    for (int kt = 0; kt < num_kt; ++kt) {
      const int s = kt % STAGES;
      if (*abort_flag || !mbar_wait(&full[s], (kt / STAGES) & 1, wait_cycles)) {
        err |= 1;
        *abort_flag = 1;
        break;
      }
      fence_after();
      const uint64_t ad = make_desc(sA + s * TILE_BYTES), bd = make_desc(sB + s * TILE_BYTES);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (BF16)
          mma_bf16(tmem, ad + (uint64_t)(k * 2), bd + (uint64_t)(k * 2), idesc, (kt | k) != 0);
        else
          mma_tf32(tmem, ad + (uint64_t)(k * 2), bd + (uint64_t)(k * 2), idesc, (kt | k) != 0);
      }
      mma_commit(&empty[s]);
    }
    mma_commit(accum);   // arrives once every MMA issued above has completed
  } else if (warp >= 2 && lane == 0) {
    if (!mbar_wait(accum, 0, wait_cycles)) {
      err |= 1;
      *abort_flag = 1;
      if (!mbar_wait(accum, 0, kDrainCycles)) err |= 2;
    }
  }
  __syncwarp();
  fence_before();
  __syncthreads();
  fence_after();
  if (warp >= 2 && !*abort_flag) {
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    const int64_t row = (int64_t)blockIdx.x * BM + q * 32 + lane;
    const double wr = (ep.mode == 0 && row < ep.M) ? ep.w[row] : 0.0;
    for (int c0 = 0; c0 < BN; c0 += 16) {
      uint32_t r[16];
      tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, r);
      tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int64_t col = (int64_t)blockIdx.y * BN + c0 + j;
        if (col >= ep.Nn) continue;
        const float v = __uint_as_float(r[j]);
        if (ep.mode == 0) {
          if (row < ep.ld_out) {
            const float z = row < ep.M ? (float)((double)v * wr) : 0.0f;
            if (ep.out_bf16)
              reinterpret_cast<__nv_bfloat16*>(ep.out)[col * ep.ld_out + row] = __float2bfloat16_rn(z);
            else
              reinterpret_cast<float*>(ep.out)[col * ep.ld_out + row] = z;
          }
        } else if (ep.mode == 1) {
          if (row < ep.M) reinterpret_cast<float*>(ep.out)[row + col * ep.ld_out] = v;
        } else {
          if (row < ep.M) reinterpret_cast<float*>(ep.out)[row * ep.ldd_m + col * ep.ldd_n] = v;
        }
      }
    }
  }
  if (err && status) atomicOr(status, (err & 2) ? (kStatTimeout | kStatDrain) : kStatTimeout);
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    tmem_dealloc(tmem, 128);
  }
}

// ---------------------------------------------------------------------------- operand copies
template <typename To>
__device__ __forceinline__ To cvt(float v);
template <> __device__ __forceinline__ float cvt<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 cvt<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// dst[c * ldd + r] = src[r * lds + c] for c < cols, r < ldd (rows r >= rows are written as 0).
template <typename To>
__global__ void k_transpose(const float* __restrict__ src, int64_t lds, int64_t rows, int64_t cols, To* __restrict__ dst,
                            int64_t ldd) {
  __shared__ float tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t r = r0 + i, c = c0 + threadIdx.x;
    tile[i][threadIdx.x] = (r < rows && c < cols) ? src[r * lds + c] : 0.0f;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t c = c0 + i, r = r0 + threadIdx.x;
    if (c < cols && r < ldd) dst[c * ldd + r] = cvt<To>(tile[threadIdx.x][i]);
  }
}

__global__ void k_to_bf16(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst, int64_t n) {
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += st) dst[i] = __float2bfloat16_rn(src[i]);
}

bool make_map(CUtensorMap* m, const void* base, bool bf16, int64_t rows, int64_t cols, int64_t ld) {
  return make_tile_map(m, base, bf16 ? 2 : 4, rows, cols, ld);
}

template <bool BF16>
cudaError_t run_gemm(const CUtensorMap& A, const CUtensorMap& B, int64_t M, int64_t Nn, int64_t K, const Epi& ep,
                     int* status, cudaStream_t s, long long wait_cycles) {
  constexpr int BK = BF16 ? 64 : 32;
  auto k = k_tc_gemm<BF16>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((M + BM - 1) / BM), (unsigned)((Nn + BN - 1) / BN));
  const int num_kt = (int)((K + BK - 1) / BK);
  k<<<grid, 192, SMEM_BYTES, s>>>(A, B, num_kt, ep, status, wait_cycles); note_launch();
  return cudaGetLastError();
}

}  // namespace

struct TcSketch {
  void* JT = nullptr;  size_t JT_bytes = 0;
  void* Jb = nullptr;  size_t Jb_bytes = 0;
  void* Ob = nullptr;  size_t Ob_bytes = 0;
  void* Zt = nullptr;  size_t Zt_bytes = 0;
};

static cudaError_t grow(void** p, size_t* cap, size_t bytes) {
  if (bytes <= *cap) return cudaSuccess;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) *cap = bytes;
  return e;
}

TcSketch* tc_create() { return new (std::nothrow) TcSketch(); }

void tc_destroy(TcSketch* t) {
  if (!t) return;
  if (t->JT) cudaFree(t->JT);
  if (t->Jb) cudaFree(t->Jb);
  if (t->Ob) cudaFree(t->Ob);
  if (t->Zt) cudaFree(t->Zt);
  delete t;
}

cudaError_t tc_sketch(TcSketch* t, bool bf16, const float* J, int64_t ldJ, int64_t N, int64_t p, const float* Omega,
                      int64_t ldY, int ell, const double* w, float* Y, const char** why, cudaStream_t s, int* status,
                      long long wait_cycles) {
  *why = nullptr;
  if (!tensor_map_encoder()) {
    *why = "cuTensorMapEncodeTiled unavailable";
    return cudaSuccess;
  }
  if ((ldJ % 32) || (ldY % 32)) {
    *why = "leading dimensions must be multiples of 32";
    return cudaSuccess;
  }
  const size_t es = bf16 ? 2 : 4;
  const int64_t ldN = (N + 31) / 32 * 32;
  cudaError_t e;
  if ((e = grow(&t->JT, &t->JT_bytes, (size_t)ldJ * ldN * es)) != cudaSuccess) return e;
  if ((e = grow(&t->Zt, &t->Zt_bytes, (size_t)ell * ldN * es)) != cudaSuccess) return e;
  // J^T (ldJ rows x ldN), zero rows beyond N handled by the transpose
  {
    dim3 blk(32, 8), grd((unsigned)((ldJ + 31) / 32), (unsigned)((ldN + 31) / 32));
    if (bf16)
      k_transpose<__nv_bfloat16><<<grd, blk, 0, s>>>(J, ldJ, N, ldJ, (__nv_bfloat16*)t->JT, ldN);
    else
      k_transpose<float><<<grd, blk, 0, s>>>(J, ldJ, N, ldJ, (float*)t->JT, ldN);
    note_launch();
  }
  const void* A1 = J;
  const void* B1 = Omega;
  if (bf16) {
    if ((e = grow(&t->Jb, &t->Jb_bytes, (size_t)N * ldJ * 2)) != cudaSuccess) return e;
    if ((e = grow(&t->Ob, &t->Ob_bytes, (size_t)ell * ldY * 2)) != cudaSuccess) return e;
    k_to_bf16<<<4096, 256, 0, s>>>(J, (__nv_bfloat16*)t->Jb, N * ldJ); note_launch();
    k_to_bf16<<<1024, 256, 0, s>>>(Omega, (__nv_bfloat16*)t->Ob, (int64_t)ell * ldY); note_launch();
    A1 = t->Jb;
    B1 = t->Ob;
  }
  CUtensorMap mA1, mB1, mA2, mB2;
  if (!make_map(&mA1, A1, bf16, N, ldJ, ldJ) || !make_map(&mB1, B1, bf16, ell, ldY, ldY) ||
      !make_map(&mA2, t->JT, bf16, ldJ, ldN, ldN) || !make_map(&mB2, t->Zt, bf16, ell, ldN, ldN)) {
    *why = "tensor map encoding failed";
    return cudaSuccess;
  }
  Epi e1{};
  e1.mode = 0;
  e1.out_bf16 = bf16 ? 1 : 0;
  e1.w = w;
  e1.out = t->Zt;
  e1.ld_out = ldN;
  e1.M = N;
  e1.Nn = ell;
  e = bf16 ? run_gemm<true>(mA1, mB1, N, ell, ldJ, e1, status, s, wait_cycles)
           : run_gemm<false>(mA1, mB1, N, ell, ldJ, e1, status, s, wait_cycles);
  if (e != cudaSuccess) return e;
  Epi e2{};
  e2.mode = 1;
  e2.out = Y;
  e2.ld_out = ldY;
  e2.M = p;
  e2.Nn = ell;
  e = bf16 ? run_gemm<true>(mA2, mB2, p, ell, ldN, e2, status, s, wait_cycles)
           : run_gemm<false>(mA2, mB2, p, ell, ldN, e2, status, s, wait_cycles);
  return e;
}

cudaError_t tc_gemm_test(bool bf16, const void* A, int64_t lda, const void* B, int64_t ldb, int64_t M, int64_t Nn,
                         int64_t K, float* D, int64_t ldd_m, int64_t ldd_n, int* status, cudaStream_t s) {
  const long long wait_cycles = kDefaultWaitCycles;
  CUtensorMap mA, mB;
  if (!make_map(&mA, A, bf16, M, K, lda) || !make_map(&mB, B, bf16, Nn, K, ldb)) return cudaErrorInvalidValue;
  Epi ep{};
  ep.mode = 2;
  ep.out = D;
  ep.M = M;
  ep.Nn = Nn;
  ep.ldd_m = ldd_m;
  ep.ldd_n = ldd_n;
  return bf16 ? run_gemm<true>(mA, mB, M, Nn, K, ep, status, s, wait_cycles)
              : run_gemm<false>(mA, mB, M, Nn, K, ep, status, s, wait_cycles);
}

}  // namespace ngd
