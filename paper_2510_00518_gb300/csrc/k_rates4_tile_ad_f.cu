// k_rates4_tile_ad_f.cu - instantiations of the tiled four-phonon kernel (float, 1-2 atoms per cell, adaptive σ).
#include "k_rates4_tile.cuh"

namespace fc4 {

cudaError_t launch4_tile_ad_f(int na, const Tables &t, const RateArgs &a, int ch, cudaStream_t s) {
    switch (na) {
    case 1: return launch4_tile<float, 1, true>(t, a, ch, s);
    case 2: return launch4_tile<float, 2, true>(t, a, ch, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace fc4
