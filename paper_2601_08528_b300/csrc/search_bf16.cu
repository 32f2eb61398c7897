// search_bf16.cu -- instantiations of the search kernel for BF16 traversal.
#include "search_kernel.cuh"

namespace svf {

cudaError_t launch_search_bf16(const SearchArgs &a, int R, int LW, bool learn, size_t smem, cudaStream_t st) {
    return launch_search_dtype<SVF_BF16, 32>(a, R, LW, learn, smem, st);
}

}  // namespace svf
