// search_u8.cu -- instantiations of the search kernel for uint8 traversal.
#include "search_kernel.cuh"

namespace svf {

cudaError_t launch_search_u8(const SearchArgs &a, int R, int LW, bool learn, size_t smem, cudaStream_t st) {
    return launch_search_dtype<SVF_U8, 64>(a, R, LW, learn, smem, st);
}

}  // namespace svf
