// search.cu -- launch of the warp-per-query search kernel (search_kernel.cuh):
// picks the instantiation for the traversal dtype, out-degree R, pool size L
// and whether the learned-stop / trace features are needed.
#include "svf_internal.h"

namespace svf {

cudaError_t launch_search_f32(const SearchArgs &a, int R, int LW, bool learn, size_t smem, cudaStream_t st);
cudaError_t launch_search_u8(const SearchArgs &a, int R, int LW, bool learn, size_t smem, cudaStream_t st);
cudaError_t launch_search_bf16(const SearchArgs &a, int R, int LW, bool learn, size_t smem, cudaStream_t st);
cudaError_t launch_search_fp8(const SearchArgs &a, int R, int LW, bool learn, size_t smem, cudaStream_t st);
cudaError_t launch_multi_f32(const SearchArgs &a, int R, int W, int LW, size_t smem, cudaStream_t st);
cudaError_t launch_multi_u8(const SearchArgs &a, int R, int W, int LW, size_t smem, cudaStream_t st);
cudaError_t launch_multi_bf16(const SearchArgs &a, int R, int W, int LW, size_t smem, cudaStream_t st);
cudaError_t launch_multi_fp8(const SearchArgs &a, int R, int W, int LW, size_t smem, cudaStream_t st);

constexpr size_t kSmemLimit = 232448;  // dynamic shared memory of one CTA (227 KB)

// The staging buffer holds one graph row's worth of candidates; the final
// re-rank stages whole primary rows (at least 4 at a time) into it and the
// visited table beside it.
size_t search_stage_bytes(const SearchArgs &a, int R) {
    size_t cap = (size_t)R * a.trav.copy_bytes;
    if (a.rerank && cap < (size_t)4 * a.prim.copy_bytes) cap = (size_t)4 * a.prim.copy_bytes;
    return cap;
}

size_t search_warp_smem(int d, int L, int R, int hash_bits, size_t stage_bytes) {
    size_t q = ((size_t)d * 4 + 15) / 16 * 16;
    size_t list = (size_t)(L > 2 * R ? L : 2 * R);
    return q + ((size_t)4 << hash_bits) + list * 4 + list * 8 + stage_bytes + 16;
}

// One CTA of W warps per query: shared query, visited table, control block
// and admitted keys (W*R), then per warp its ids, keys and staging buffer.
// The staging buffer shrinks (rows are then staged in several rounds) when
// W full-size buffers do not fit; it keeps room for one row of each store
// it reads.
size_t search_multi_smem(SearchArgs &a, int W, int R) {
    const size_t fixed = (size_t)a.q_bytes + ((size_t)4 << a.hash_bits) + kMultiCtlBytes + (size_t)W * R * 8;
    const size_t lists = (size_t)a.list_len * 12 + 16;
    size_t stage = a.stage_bytes;
    if (fixed + (size_t)W * (lists + stage) > kSmemLimit) {
        const size_t room = kSmemLimit > fixed + (size_t)W * lists ? (kSmemLimit - fixed) / W - lists : 0;
        stage = room / 16 * 16;
        size_t need = a.trav.copy_bytes;
        if (a.rerank && (size_t)a.prim.copy_bytes > need) need = a.prim.copy_bytes;
        if (stage < need) return 0;
    }
    a.stage_bytes = (uint32_t)stage;
    a.warp_smem = lists + stage;
    return fixed + (size_t)W * a.warp_smem;
}

cudaError_t launch_search(SearchArgs a, int R, int L, cudaStream_t st) {
    a.list_len = L > 2 * R ? L : 2 * R;
    a.stage_bytes = (uint32_t)search_stage_bytes(a, R);
    if (a.W > 1) {
        const size_t smem = search_multi_smem(a, a.W, R);
        if (smem == 0) return cudaErrorInvalidValue;
        const int LW = L / 32;
        switch (a.trav.dtype) {
        case SVF_F32: return launch_multi_f32(a, R, a.W, LW, smem, st);
        case SVF_U8: return launch_multi_u8(a, R, a.W, LW, smem, st);
        case SVF_BF16: return launch_multi_bf16(a, R, a.W, LW, smem, st);
        default: return launch_multi_fp8(a, R, a.W, LW, smem, st);
        }
    }
    a.warp_smem = search_warp_smem(a.trav.d, L, R, a.hash_bits, a.stage_bytes);
    const size_t smem = a.warp_smem * kSearchWarps;
    const int LW = L / 32;
    const bool learn = a.mlp != nullptr || a.trace_feat != nullptr;
    switch (a.trav.dtype) {
    case SVF_F32: return launch_search_f32(a, R, LW, learn, smem, st);
    case SVF_U8: return launch_search_u8(a, R, LW, learn, smem, st);
    case SVF_BF16: return launch_search_bf16(a, R, LW, learn, smem, st);
    default: return launch_search_fp8(a, R, LW, learn, smem, st);
    }
}

}  // namespace svf
