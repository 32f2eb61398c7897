// search_fp8.cu -- instantiations of the search kernel for FP8-E4M3 traversal.
#include "search_kernel.cuh"

namespace svf {

namespace {
template <int R, bool LEARN>
cudaError_t go(const SearchArgs &a, int LW, size_t smem, cudaStream_t st) {
    dim3 grid((unsigned)((a.nq + kSearchWarps - 1) / kSearchWarps)), block(kSearchWarps * 32);
    switch (LW) {
#define SVF_LW_CASE(X)                                                                                        \
    case X:                                                                                                   \
        if (cudaFuncSetAttribute(search_kernel<SVF_FP8, R, X, LEARN>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 (int)smem) != cudaSuccess)                                                   \
            return cudaGetLastError();                                                                        \
        search_kernel<SVF_FP8, R, X, LEARN><<<grid, block, smem, st>>>(a);                                       \
        return cudaGetLastError();
        SVF_LW_CASE(1)
        SVF_LW_CASE(2)
        SVF_LW_CASE(4)
        SVF_LW_CASE(8)
#undef SVF_LW_CASE
    }
    return cudaErrorInvalidValue;
}
}  // namespace

cudaError_t launch_search_fp8(const SearchArgs &a, int R, int LW, bool learn, size_t smem, cudaStream_t st) {
    if (R == 32) return learn ? go<32, true>(a, LW, smem, st) : go<32, false>(a, LW, smem, st);
    return learn ? go<64, true>(a, LW, smem, st) : go<64, false>(a, LW, smem, st);
}

}  // namespace svf
