// The double-float GEMM instantiated for float A and float B operands (templates in gemm_df.cuh).
#include "gemm_df.cuh"

namespace ngd {

template void launch_gemm_df<float, float>(const GemmDfArgs<float, float>&, cudaStream_t);

}  // namespace ngd
