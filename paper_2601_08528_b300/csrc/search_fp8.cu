// search_fp8.cu -- instantiations of the search kernel for FP8-E4M3 traversal.
#include "search_multi.cuh"

namespace svf {

cudaError_t launch_search_fp8(const SearchArgs &a, int R, int LW, bool learn, size_t smem, cudaStream_t st) {
    return launch_search_dtype<SVF_FP8, 32>(a, R, LW, learn, smem, st);
}

cudaError_t launch_multi_fp8(const SearchArgs &a, int R, int W, int LW, size_t smem, cudaStream_t st) {
    return launch_multi_dtype<SVF_FP8, 32>(a, R, W, LW, smem, st);
}

}  // namespace svf
