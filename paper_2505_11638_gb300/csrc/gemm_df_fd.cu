// The double-float GEMM instantiated for float A and double B operands (templates in gemm_df.cuh).
#include "gemm_df.cuh"

namespace ngd {

template void launch_gemm_df<float, double>(const GemmDfArgs<float, double>&, cudaStream_t);

}  // namespace ngd
