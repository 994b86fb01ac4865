// Delay-and-sum energy image (Eq. 1 + Eq. 3; multistatic: Eq. 2 + Eq. 4).
// Instantiations of the image kernel for DAS, one instance per window chunk WT, monostatic and multistatic.
#include "image_common.cuh"

namespace uwb {

cudaError_t launch_image_das(int v, bool ms, const ImgParams& p, const CUtensorMap* tmap,
                               int ctas, int threads, size_t smem, cudaStream_t st) {
  switch (v) {
    case 4:
      return ms ? launch_variant<BF_DAS, 4, true>(p, tmap, ctas, threads, smem, st)
                : launch_variant<BF_DAS, 4, false>(p, tmap, ctas, threads, smem, st);
    case 8:
      return ms ? launch_variant<BF_DAS, 8, true>(p, tmap, ctas, threads, smem, st)
                : launch_variant<BF_DAS, 8, false>(p, tmap, ctas, threads, smem, st);
    case 16:
      return ms ? launch_variant<BF_DAS, 16, true>(p, tmap, ctas, threads, smem, st)
                : launch_variant<BF_DAS, 16, false>(p, tmap, ctas, threads, smem, st);
    case 20:
      return ms ? launch_variant<BF_DAS, 20, true>(p, tmap, ctas, threads, smem, st)
                : launch_variant<BF_DAS, 20, false>(p, tmap, ctas, threads, smem, st);
    case 32:  // multistatic only (monostatic windows over 20 go in chunks of 16)
      return ms ? launch_variant<BF_DAS, 32, true>(p, tmap, ctas, threads, smem, st)
                : cudaErrorInvalidValue;
    default:
      return cudaErrorInvalidValue;
  }
}

int occupancy_image_das(int v, bool ms, bool rg, int threads, size_t smem) {
  switch (v) {
    case 4:
      return ms ? occupancy_variant<BF_DAS, 4, true>(rg, threads, smem)
                : occupancy_variant<BF_DAS, 4, false>(rg, threads, smem);
    case 8:
      return ms ? occupancy_variant<BF_DAS, 8, true>(rg, threads, smem)
                : occupancy_variant<BF_DAS, 8, false>(rg, threads, smem);
    case 16:
      return ms ? occupancy_variant<BF_DAS, 16, true>(rg, threads, smem)
                : occupancy_variant<BF_DAS, 16, false>(rg, threads, smem);
    case 20:
      return ms ? occupancy_variant<BF_DAS, 20, true>(rg, threads, smem)
                : occupancy_variant<BF_DAS, 20, false>(rg, threads, smem);
    case 32:
      return ms ? occupancy_variant<BF_DAS, 32, true>(rg, threads, smem) : 0;
    default:
      return 0;
  }
}

}  // namespace uwb
