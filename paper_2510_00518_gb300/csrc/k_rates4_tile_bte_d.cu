// k_rates4_tile_bte_d.cu - instantiations of the tiled four-phonon kernel that also accumulate the
// iterative Boltzmann equation's off-diagonal term (double, 1-2 atoms per cell, fixed and adaptive σ).
#include "k_rates4_tile.cuh"

namespace fc4 {

cudaError_t launch4_tile_bte_d(int na, const Tables &t, const RateArgs &a, int ch, cudaStream_t s) {
    const bool ad = a.adaptive != 0;
    switch (na) {
    case 1: return ad ? launch4_tile<double, 1, true, true>(t, a, ch, s) : launch4_tile<double, 1, false, true>(t, a, ch, s);
    case 2: return ad ? launch4_tile<double, 2, true, true>(t, a, ch, s) : launch4_tile<double, 2, false, true>(t, a, ch, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace fc4
