// FP64-accurate Nystrom sketch Y = J^T diag(w) (J Omega) on the tcgen05 tensor cores by an
// error-free split of the operands into BF16 digit planes (sketch_oz.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ngd {

struct OzSketch;   // digit planes of J (per linearization), of Omega and Z, split-K partials

OzSketch* oz_create();
void oz_destroy(OzSketch* o);

// Y64 (p x ell, column-major, leading dimension ldY, float64) = J^T diag(w) J Omega for the FP32
// Jacobian J (N x ldJ row-major, zero columns p..ldJ-1) and the FP32 test matrix Omega (p x ell,
// column-major, leading dimension ldY, zero rows p..ldY-1).  j_version identifies the contents
// of J: the digit planes of J are rebuilt when it changes.  Accuracy: every kept digit product
// is summed exactly; the dropped digit products and the rounded low levels leave ~2^-46 of the
// term magnitudes.  On a configuration it cannot serve it sets *why and returns cudaSuccess
// without work.  A device-side wait that ran out sets kStatTimeout in *status.
cudaError_t oz_sketch(OzSketch* o, const float* J, int64_t ldJ, int64_t N, int64_t p, uint64_t j_version,
                      const float* Omega, int64_t ldY, int ell, const double* w, double* Y64, const char** why,
                      cudaStream_t s, int* status, long long wait_cycles);

// Lower triangle (entries m >= n) of G (p x p, column-major, leading dimension ldG >= p, float64)
// = J^T diag(w) J for the FP32 Jacobian J (N x ldJ row-major, zero columns p..ldJ-1): NGD full's
// Gramian by the same digit-plane tensor-core GEMM, with J^T and (diag(w) J)^T split per column
// of J into six digits each (pairs with s + t <= 5 kept; ~2^-46 of the term magnitudes).  Entries
// m < n are left untouched (the caller mirrors the lower triangle).  *why / status as oz_sketch.
cudaError_t oz_gram(OzSketch* o, const float* J, int64_t ldJ, int64_t N, int64_t p, const double* w, double* G,
                    int64_t ldG, const char** why, cudaStream_t s, int* status, long long wait_cycles);

// Lower triangle (entries m >= n) of C (ell x ell, column-major, leading dimension ldC, float64) =
// A^T B for the column-major K x ell operands A and B (leading dimension ld, a multiple of 32;
// rows K..ld-1 are not read): A = A32 (FP32, five digits per column) or, with A32 null, A = B
// (B^T B); B in FP64 with six digits per column.  The Nystrom factor's Omega^T Y_nu and B^T B on
// the digit-plane tensor-core GEMM, accurate to ~2^-46 of the products of the columns' largest
// entries per term.  Entries m < n are left untouched.  *why / status as oz_sketch.
cudaError_t oz_gram_cols(OzSketch* o, const float* A32, const double* B, int64_t K, int64_t ld, int ell, double* C,
                         int64_t ldC, const char** why, cudaStream_t s, int* status, long long wait_cycles);

// U (p x ell, column-major, leading dimension ldU >= p, float64; rows p..ldU-1 written as zero) =
// B W diag(colscale) for the FP64 operands B (p x ell, column-major, leading dimension ldB) and W
// (ell x ell, column-major, leading dimension ldW): the Nystrom factor's U = B V Sigma^-1 on the
// digit-plane tensor-core GEMM, B split per row and W diag(colscale) per column into six digits
// each (~2^-46 of the products of a row's and a column's largest entries per term).  *why /
// status as oz_sketch.
// Lower triangle (entries m >= n) of C (ell x ell, float64) = A^T A for the FP32 column-major
// K x ell A (leading dimension ld, a multiple of 32; rows K..ld-1 not read), five digits per
// column: the CholeskyQR Gram matrix of the test matrix, FP64-accurate.  Entries m < n are left
// untouched.  *why / status as oz_sketch.
cudaError_t oz_gram_self32(OzSketch* o, const float* A, int64_t K, int64_t ld, int ell, double* C, int64_t ldC,
                           const char** why, cudaStream_t s, int* status, long long wait_cycles);

// Lower triangle (entries m >= n) of C (m x m, column-major, leading dimension ldC, float64) -=
// P P^T for the FP64 panel P (m x bs, column-major, leading dimension ldP, bs <= 256): the trailing
// update of a blocked Cholesky on the digit-plane tensor-core GEMM, P split per row into six
// digits (~2^-46 of the products of two rows' largest entries per term), one K chunk, the scaled
// product subtracted by the GEMM's epilogue.  Entries m < n are left untouched.  *why / status as
// oz_sketch.
cudaError_t oz_syrk_sub(OzSketch* o, const double* P, int64_t ldP, int64_t m, int bs, double* C, int64_t ldC,
                        const char** why, cudaStream_t s, int* status, long long wait_cycles);

cudaError_t oz_gemm_bw(OzSketch* o, const double* B, int64_t ldB, int64_t p, int ell, const double* W, int64_t ldW,
                       const double* colscale, double* U, int64_t ldU, const char** why, cudaStream_t s, int* status,
                       long long wait_cycles);

}  // namespace ngd
