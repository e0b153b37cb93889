// k_rates4_tile_d.cu - instantiations of the tiled four-phonon kernel (double, 1-2 atoms per cell, fixed σ).
#include "k_rates4_tile.cuh"

namespace fc4 {

cudaError_t launch4_tile_d(int na, const Tables &t, const RateArgs &a, int ch, cudaStream_t s) {
    switch (na) {
    case 1: return launch4_tile<double, 1, false>(t, a, ch, s);
    case 2: return launch4_tile<double, 2, false>(t, a, ch, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace fc4
