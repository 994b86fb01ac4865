// Delay-and-sum energy image (Eq. 1 + Eq. 3).
// Instantiations of the image kernel for DAS, one instance per window chunk WT.
#include "image_common.cuh"

namespace uwb {

cudaError_t launch_image_das(int v, const ImgParams& p, const CUtensorMap* tmap, int ctas,
                               int threads, size_t smem, cudaStream_t st) {
  switch (v) {
    case 4:
      return launch_variant<BF_DAS, 4>(p, tmap, ctas, threads, smem, st);
    case 8:
      return launch_variant<BF_DAS, 8>(p, tmap, ctas, threads, smem, st);
    case 16:
      return launch_variant<BF_DAS, 16>(p, tmap, ctas, threads, smem, st);
    case 20:
      return launch_variant<BF_DAS, 20>(p, tmap, ctas, threads, smem, st);
    case 32:
      return launch_variant<BF_DAS, 32>(p, tmap, ctas, threads, smem, st);
    default:
      return cudaErrorInvalidValue;
  }
}

int occupancy_image_das(int v, int threads, size_t smem) {
  switch (v) {
    case 4:
      return occupancy_variant<BF_DAS, 4>(threads, smem);
    case 8:
      return occupancy_variant<BF_DAS, 8>(threads, smem);
    case 16:
      return occupancy_variant<BF_DAS, 16>(threads, smem);
    case 20:
      return occupancy_variant<BF_DAS, 20>(threads, smem);
    case 32:
      return occupancy_variant<BF_DAS, 32>(threads, smem);
    default:
      return 0;
  }
}

}  // namespace uwb
