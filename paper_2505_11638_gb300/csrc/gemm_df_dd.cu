// The double-float GEMM instantiated for double A and double B operands (templates in gemm_df.cuh).
#include "gemm_df.cuh"

namespace ngd {

template void launch_gemm_df<double, double>(const GemmDfArgs<double, double>&, cudaStream_t);

}  // namespace ngd
