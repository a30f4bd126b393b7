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

// G (p x p, column-major, leading dimension ldG >= p, float64) = J^T diag(w) J for the FP32
// Jacobian J (N x ldJ row-major, zero columns p..ldJ-1): NGD full's Gramian by the same digit-plane
// tensor-core GEMM, with J^T and (diag(w) J)^T split per column of J into six digits each (pairs
// with s + t <= 5 kept; ~2^-46 of the term magnitudes).  Every entry of G is written (the upper
// triangle is the transposed product, equal up to rounding).  *why / status as oz_sketch.
cudaError_t oz_gram(OzSketch* o, const float* J, int64_t ldJ, int64_t N, int64_t p, const double* w, double* G,
                    int64_t ldG, const char** why, cudaStream_t s, int* status, long long wait_cycles);

}  // namespace ngd
