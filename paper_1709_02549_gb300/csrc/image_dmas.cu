// Delay-multiply-and-sum energy image (Section II.B), pair sum through the
// identity sum_{i<j} x_i x_j = ((sum x)^2 - sum x^2) / 2.
// Instantiations of the image kernel for DMAS (identity form), one instance per window chunk WT.
#include "image_common.cuh"

namespace uwb {

cudaError_t launch_image_dmas(int v, const ImgParams& p, const CUtensorMap* tmap, int ctas,
                               int threads, size_t smem, cudaStream_t st) {
  switch (v) {
    case 4:
      return launch_variant<BF_DMAS_ID, 4>(p, tmap, ctas, threads, smem, st);
    case 8:
      return launch_variant<BF_DMAS_ID, 8>(p, tmap, ctas, threads, smem, st);
    case 16:
      return launch_variant<BF_DMAS_ID, 16>(p, tmap, ctas, threads, smem, st);
    case 20:
      return launch_variant<BF_DMAS_ID, 20>(p, tmap, ctas, threads, smem, st);
    case 32:
      return launch_variant<BF_DMAS_ID, 32>(p, tmap, ctas, threads, smem, st);
    default:
      return cudaErrorInvalidValue;
  }
}

int occupancy_image_dmas(int v, int threads, size_t smem) {
  switch (v) {
    case 4:
      return occupancy_variant<BF_DMAS_ID, 4>(threads, smem);
    case 8:
      return occupancy_variant<BF_DMAS_ID, 8>(threads, smem);
    case 16:
      return occupancy_variant<BF_DMAS_ID, 16>(threads, smem);
    case 20:
      return occupancy_variant<BF_DMAS_ID, 20>(threads, smem);
    case 32:
      return occupancy_variant<BF_DMAS_ID, 32>(threads, smem);
    default:
      return 0;
  }
}

}  // namespace uwb
