// Search kernels for one plane layout (5 bit planes of uint32_t words), thresholds 2..8.
#include "pms_search.cuh"

namespace pms {

cudaError_t launch_search_p5_32(int t, const SearchArgs &a, cudaStream_t s)
{
    return search::launch_layout<5, uint32_t>(t, a, s);
}

int max_blocks_p5_32(int t, int wpb)
{
    return search::max_blocks_layout<5, uint32_t>(t, wpb);
}

size_t fscr_p5_32(int lmax)
{
    return search::fscr_layout<5, uint32_t>(lmax);
}

}  // namespace pms
