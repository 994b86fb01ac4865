// Delay-multiply-and-sum energy image (Section II.B) with every antenna pair
// multiplied explicitly.
// Instantiations of the image kernel for literal-pair DMAS, one instance per antenna register block MMAX.
#include "image_common.cuh"

namespace uwb {

cudaError_t launch_image_literal(int v, const ImgParams& p, const CUtensorMap* tmap,
                               int ctas, int threads, size_t smem, cudaStream_t st) {
  switch (v) {
    case 16:
      return launch_variant<BF_DMAS_LIT, 16, false>(p, tmap, ctas, threads, smem, st);
    case 32:
      return launch_variant<BF_DMAS_LIT, 32, false>(p, tmap, ctas, threads, smem, st);
    case 64:
      return launch_variant<BF_DMAS_LIT, 64, false>(p, tmap, ctas, threads, smem, st);
    case 96:
      return launch_variant<BF_DMAS_LIT, 96, false>(p, tmap, ctas, threads, smem, st);
    default:
      return cudaErrorInvalidValue;
  }
}

int occupancy_image_literal(int v, bool rg, int threads, size_t smem) {
  switch (v) {
    case 16:
      return occupancy_variant<BF_DMAS_LIT, 16, false>(rg, threads, smem);
    case 32:
      return occupancy_variant<BF_DMAS_LIT, 32, false>(rg, threads, smem);
    case 64:
      return occupancy_variant<BF_DMAS_LIT, 64, false>(rg, threads, smem);
    case 96:
      return occupancy_variant<BF_DMAS_LIT, 96, false>(rg, threads, smem);
    default:
      return 0;
  }
}

}  // namespace uwb
