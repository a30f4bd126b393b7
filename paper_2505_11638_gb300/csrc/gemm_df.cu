// The double-float GEMM's K-slice rule, and its (double, float) instantiation; the templates are in
// gemm_df.cuh.
#include "gemm_df.cuh"

namespace ngd {

// K slices for the vectorised double-float GEMM on an M x N output: the count (at most 32, each
// slice at least 128 deep) whose blocks fill the resident block slots (2 per SM) most evenly.
// lower: only the tiles of the lower triangle run (the others return at once), so only they count.
int gemm_df_splits(int64_t M, int64_t N, int64_t K, bool lower) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t slots = 2 * (int64_t)std::max(sms, 1);
  const int64_t tn = N <= gdf::BN / 2 ? gdf::BN / 2 : gdf::BN;   // the 32-wide tile of skinny FP64 B
  const int64_t mt = (M + gdf::BM - 1) / gdf::BM, nt = (N + tn - 1) / tn;
  int64_t tiles = mt * nt;
  if (lower) {
    tiles = 0;
    for (int64_t a = 0; a < mt; ++a) tiles += std::min<int64_t>(nt, (gdf::BM * (a + 1) + tn - 1) / tn);
  }
  int best = 1;
  double best_eff = 0.0;
  for (int ns = 1; ns <= 32 && (ns == 1 || K / ns >= 128); ++ns) {
    const int64_t blocks = tiles * ns;
    const int64_t waves = (blocks + slots - 1) / slots;
    const double eff = (double)blocks / (double)(waves * slots);
    if (eff > best_eff + 0.02) {
      best_eff = eff;
      best = ns;
    }
  }
  return best;
}

template void launch_gemm_df<double, float>(const GemmDfArgs<double, float>&, cudaStream_t);

}  // namespace ngd
