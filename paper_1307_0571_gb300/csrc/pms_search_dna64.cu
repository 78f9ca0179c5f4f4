// Search kernels for one plane layout (2 bit planes of uint64_t words), thresholds 2..8.
// Index checks stay on for the 64-bit-plane layouts: a (50,21) run of this layout returned
// a CUDA error that a checked build of the same run did not reproduce.
#ifndef PMS_BOUNDS_CHECK
#define PMS_BOUNDS_CHECK 1
#endif
#include "pms_search.cuh"

namespace pms {

cudaError_t launch_search_dna64(int t, const SearchArgs &a, cudaStream_t s)
{
    return search::launch_layout<2, uint64_t>(t, a, s);
}

int max_blocks_dna64(int t, int wpb)
{
    return search::max_blocks_layout<2, uint64_t>(t, wpb);
}

size_t fscr_dna64(int lmax)
{
    return search::fscr_layout<2, uint64_t>(lmax);
}

}  // namespace pms
