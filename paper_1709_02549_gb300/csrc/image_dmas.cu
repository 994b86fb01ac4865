// Delay-multiply-and-sum energy image (Section II.B), pair sum through the
// identity sum_{i<j} x_i x_j = ((sum x)^2 - sum x^2) / 2.
// Instantiations of the image kernel for DMAS (identity form), one instance per window chunk WT, monostatic and
// multistatic.
#include "image_common.cuh"

namespace uwb {

cudaError_t launch_image_dmas(int v, bool ms, const ImgParams& p, const CUtensorMap* tmap,
                               int ctas, int threads, size_t smem, cudaStream_t st) {
  switch (v) {
    case 4:
      return ms ? launch_variant<BF_DMAS_ID, 4, true>(p, tmap, ctas, threads, smem, st)
                : launch_variant<BF_DMAS_ID, 4, false>(p, tmap, ctas, threads, smem, st);
    case 8:
      return ms ? launch_variant<BF_DMAS_ID, 8, true>(p, tmap, ctas, threads, smem, st)
                : launch_variant<BF_DMAS_ID, 8, false>(p, tmap, ctas, threads, smem, st);
    case 16:
      return ms ? launch_variant<BF_DMAS_ID, 16, true>(p, tmap, ctas, threads, smem, st)
                : launch_variant<BF_DMAS_ID, 16, false>(p, tmap, ctas, threads, smem, st);
    case 20:
      return ms ? launch_variant<BF_DMAS_ID, 20, true>(p, tmap, ctas, threads, smem, st)
                : launch_variant<BF_DMAS_ID, 20, false>(p, tmap, ctas, threads, smem, st);
    case 32:  // multistatic only (monostatic windows over 20 go in chunks of 16)
      return ms ? launch_variant<BF_DMAS_ID, 32, true>(p, tmap, ctas, threads, smem, st)
                : cudaErrorInvalidValue;
    default:
      return cudaErrorInvalidValue;
  }
}

int occupancy_image_dmas(int v, bool ms, bool rg, int threads, size_t smem) {
  switch (v) {
    case 4:
      return ms ? occupancy_variant<BF_DMAS_ID, 4, true>(rg, threads, smem)
                : occupancy_variant<BF_DMAS_ID, 4, false>(rg, threads, smem);
    case 8:
      return ms ? occupancy_variant<BF_DMAS_ID, 8, true>(rg, threads, smem)
                : occupancy_variant<BF_DMAS_ID, 8, false>(rg, threads, smem);
    case 16:
      return ms ? occupancy_variant<BF_DMAS_ID, 16, true>(rg, threads, smem)
                : occupancy_variant<BF_DMAS_ID, 16, false>(rg, threads, smem);
    case 20:
      return ms ? occupancy_variant<BF_DMAS_ID, 20, true>(rg, threads, smem)
                : occupancy_variant<BF_DMAS_ID, 20, false>(rg, threads, smem);
    case 32:
      return ms ? occupancy_variant<BF_DMAS_ID, 32, true>(rg, threads, smem) : 0;
    default:
      return 0;
  }
}

}  // namespace uwb
