// Tensor-core (tcgen05 + TMA) Nystrom sketch Y = J^T diag(w) (J Omega).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ngd {

struct TcSketch;  // operand copies (transposed / BF16 Jacobian, Z^T) and tensor maps

TcSketch* tc_create();
void tc_destroy(TcSketch* t);

// Y (ldY x ell, column-major, FP32) = J^T diag(w) J Omega with J (N x ldJ, row-major FP32,
// zero columns p..ldJ-1) and Omega (ldY x ell column-major FP32, zero rows p..ldY-1).
// bf16 selects BF16 operands (round to nearest), else TF32 (FP32 bits read by the tensor
// core).  Accumulation is FP32 in tensor memory.  On a configuration it cannot serve it
// sets *why and returns cudaSuccess without work; a device-side wait that ran out sets the
// status word bit kStatTimeout in *status (nullable).
// wait_cycles: clock limit of each bounded mbarrier wait (tc_common.cuh).
cudaError_t tc_sketch(TcSketch* t, bool bf16, const float* J, int64_t ldJ, int64_t N, int64_t p, const float* Omega,
                      int64_t ldY, int ell, const double* w, float* Y, const char** why, cudaStream_t s,
                      int* status, long long wait_cycles);

// Plain tcgen05 GEMM D = A B^T (both K-major), exposed for tests: A (M x K, lda), B (Nn x K, ldb),
// FP32 or BF16 operands, D (M x Nn) written as D[m*ldd_m + n*ldd_n] in FP32.
cudaError_t tc_gemm_test(bool bf16, const void* A, int64_t lda, const void* B, int64_t ldb, int64_t M, int64_t Nn,
                         int64_t K, float* D, int64_t ldd_m, int64_t ldd_n, int* status, cudaStream_t s);

}  // namespace ngd
