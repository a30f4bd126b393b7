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
// drain it with tcgen05.ld.  Every mbarrier wait is bounded by a clock deadline; on
// expiry the kernel records kStatTimeout, finishes its own bookkeeping, frees its TMEM
// and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "ngd_internal.cuh"
#include "sketch_tc.cuh"

namespace ngd {

namespace {

constexpr int BM = 128, BN = 128, STAGES = 6;
constexpr int TILE_BYTES = 128 * 128;                    // 128 rows x 128 bytes
constexpr int SMEM_BYTES = 2 * STAGES * TILE_BYTES + 1024 + 256;
constexpr long long kWaitCycles = 4000000000ll;          // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t cnt) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(cnt) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: true when the phase with the given parity completed, false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(b, parity)) {
    if (clock64() - t0 > kWaitCycles) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor, K-major, 128-byte swizzle: start >> 4, LBO (unused for this
// layout, 16 B), SBO = 1024 B between 8-row groups, descriptor version 1, layout type 2.
__device__ __forceinline__ uint64_t make_desc(const void* p) {
  const uint64_t a = smem_u32(p);
  return ((a & 0x3FFFFull) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) |
         ((uint64_t)2 << 61);
}

// Instruction descriptor: D FP32, A/B format (TF32 = 2 for kind::tf32, BF16 = 1 for kind::f16),
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t make_idesc(uint32_t fmt, uint32_t m, uint32_t n) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((n >> 3) << 17) | ((m >> 4) << 24);
}

template <bool BF16>
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if (BF16) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

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
                                                   int* status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * TILE_BYTES;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + 2 * STAGES * TILE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* accum = empty + STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accum, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(128)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  bool err = false;

  if (warp == 0 && lane == 0) {
    const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
    constexpr int BK = BF16 ? 64 : 32;
    for (int kt = 0; kt < num_kt; ++kt) {
      const int s = kt % STAGES;
      if (kt >= STAGES && !mbar_wait(&empty[s], ((kt / STAGES) - 1) & 1)) {
        err = true;
        break;
      }
      mbar_expect_tx(&full[s], 2 * TILE_BYTES);
      tma_load_2d(sA + s * TILE_BYTES, &tmA, kt * BK, m0, &full[s]);
      tma_load_2d(sB + s * TILE_BYTES, &tmB, kt * BK, n0, &full[s]);
    }
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = make_idesc(BF16 ? 1u : 2u, BM, BN);
    for (int kt = 0; kt < num_kt; ++kt) {
      const int s = kt % STAGES;
      if (!mbar_wait(&full[s], (kt / STAGES) & 1)) {
        err = true;
        break;
      }
      tc_fence_after();
      const uint64_t ad = make_desc(sA + s * TILE_BYTES), bd = make_desc(sB + s * TILE_BYTES);
#pragma unroll
      for (int k = 0; k < 4; ++k) mma<BF16>(tmem, ad + (uint64_t)(k * 2), bd + (uint64_t)(k * 2), idesc, (kt | k) != 0);
      mma_commit(&empty[s]);
    }
    mma_commit(accum);
  } else if (warp >= 2) {
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    if (!mbar_wait(accum, 0)) {
      err = true;
    } else {
      tc_fence_after();
      const int64_t row = (int64_t)blockIdx.x * BM + q * 32 + lane;
      const double wr = (ep.mode == 0 && row < ep.M) ? ep.w[row] : 0.0;
      for (int c0 = 0; c0 < BN; c0 += 16) {
        uint32_t r[16];
        tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, r);
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
  }
  if (err && status) atomicOr(status, kStatTimeout);
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128) : "memory");
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

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn get_encode() {
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

// 2-D row-major map: rows x cols (cols contiguous, row stride ld elements), box 128 rows x 128 bytes.
bool make_map(CUtensorMap* m, const void* base, bool bf16, int64_t rows, int64_t cols, int64_t ld) {
  EncodeFn enc = get_encode();
  if (!enc) return false;
  const size_t es = bf16 ? 2 : 4;
  if ((reinterpret_cast<uintptr_t>(base) & 15) || ((ld * es) & 15)) return false;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * es)};
  cuuint32_t box[2] = {(cuuint32_t)(128 / es), 128u};
  cuuint32_t estr[2] = {1u, 1u};
  const CUresult r = enc(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                         const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <bool BF16>
cudaError_t run_gemm(const CUtensorMap& A, const CUtensorMap& B, int64_t M, int64_t Nn, int64_t K, const Epi& ep,
                     int* status, cudaStream_t s) {
  constexpr int BK = BF16 ? 64 : 32;
  auto k = k_tc_gemm<BF16>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((M + BM - 1) / BM), (unsigned)((Nn + BN - 1) / BN));
  const int num_kt = (int)((K + BK - 1) / BK);
  k<<<grid, 192, SMEM_BYTES, s>>>(A, B, num_kt, ep, status); note_launch();
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
                      int64_t ldY, int ell, const double* w, float* Y, const char** why, cudaStream_t s, int* status) {
  *why = nullptr;
  if (!get_encode()) {
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
  e = bf16 ? run_gemm<true>(mA1, mB1, N, ell, ldJ, e1, status, s) : run_gemm<false>(mA1, mB1, N, ell, ldJ, e1, status, s);
  if (e != cudaSuccess) return e;
  Epi e2{};
  e2.mode = 1;
  e2.out = Y;
  e2.ld_out = ldY;
  e2.M = p;
  e2.Nn = ell;
  e = bf16 ? run_gemm<true>(mA2, mB2, p, ell, ldN, e2, status, s) : run_gemm<false>(mA2, mB2, p, ell, ldN, e2, status, s);
  return e;
}

cudaError_t tc_gemm_test(bool bf16, const void* A, int64_t lda, const void* B, int64_t ldb, int64_t M, int64_t Nn,
                         int64_t K, float* D, int64_t ldd_m, int64_t ldd_n, int* status, cudaStream_t s) {
  CUtensorMap mA, mB;
  if (!make_map(&mA, A, bf16, M, K, lda) || !make_map(&mB, B, bf16, Nn, K, ldb)) return cudaErrorInvalidValue;
  Epi ep{};
  ep.mode = 2;
  ep.out = D;
  ep.M = M;
  ep.Nn = Nn;
  ep.ldd_m = ldd_m;
  ep.ldd_n = ldd_n;
  return bf16 ? run_gemm<true>(mA, mB, M, Nn, K, ep, status, s) : run_gemm<false>(mA, mB, M, Nn, K, ep, status, s);
}

}  // namespace ngd
