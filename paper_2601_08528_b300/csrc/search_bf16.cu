// search_bf16.cu -- instantiations of the search kernel for BF16 traversal.
#include "search_multi.cuh"

namespace svf {

cudaError_t launch_search_bf16(const SearchArgs &a, int R, int LW, bool learn, size_t smem, cudaStream_t st) {
    return launch_search_dtype<SVF_BF16, 32>(a, R, LW, learn, smem, st);
}

cudaError_t launch_multi_bf16(const SearchArgs &a, int R, int W, int LW, size_t smem, cudaStream_t st) {
    return launch_multi_dtype<SVF_BF16, 32>(a, R, W, LW, smem, st);
}

}  // namespace svf
