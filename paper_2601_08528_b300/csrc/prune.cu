// prune.cu -- neighbour reordering of a sorted candidate list (SVFusion
// Sec. 5.1): every candidate c_i gets a detour count, the list is stably
// sorted by ascending count and the first R are kept.
//   RNG  count_i = #{ j < i : dist(c_j, c_i) < dist(v, c_i) }
//   RANK count_i = #{ j < i : c_i in N_out(c_j) }   (no distances)
// One CTA per candidate list.  RNG stages the candidate rows in shared
// memory when they fit and evaluates the m(m-1)/2 pairs with teams of 8
// lanes; RANK maps ids to positions with a shared-memory hash.  The stable
// sort is a rank computation on (count, position).
#include <cstdint>

#include "svf_internal.h"

namespace svf {

namespace {
constexpr int THREADS = 256;
constexpr int MAXC = 512;

__device__ __forceinline__ void pair_of(int p, int &i, int &j) {
    // p enumerates pairs (i, j), j < i, in order of i: p = i(i-1)/2 + j
    int t = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)p)) * 0.5f);
    while (t * (t - 1) / 2 > p) t--;
    while ((t + 1) * t / 2 <= p) t++;
    i = t;
    j = p - t * (t - 1) / 2;
}

template <int DT>
__global__ void __launch_bounds__(THREADS) prune_kernel(const PruneArgs a, int stage) {
    extern __shared__ __align__(16) uint8_t sm[];
    uint32_t *ids = reinterpret_cast<uint32_t *>(sm);
    uint32_t *dk = ids + MAXC;
    int *cnt = reinterpret_cast<int *>(dk + MAXC);
    uint32_t *hkey = reinterpret_cast<uint32_t *>(cnt + MAXC);  // RANK: 2*MAXC slots
    int *hpos = reinterpret_cast<int *>(hkey + 2 * MAXC);
    uint4 *rows = reinterpret_cast<uint4 *>(hpos + 2 * MAXC);  // staged rows (RNG)

    const int tid = threadIdx.x, lane = tid & 31, team = tid >> 3, sub = tid & 7;
    const int nteams = THREADS / kTeam;
    const int64_t nlists = a.count ? (int64_t)*a.count : a.nv;
    for (int64_t li = blockIdx.x; li < nlists; li += gridDim.x) {
        const uint64_t *kl = a.cand + li * a.cand_stride;
        int mloc = 0;
        for (int i = tid; i < a.cand_stride && i < MAXC; i += THREADS) {
            uint64_t k = kl[i];
            bool real = !key_is_pad(k);
            ids[i] = real ? key_id(k) : kEmpty;
            dk[i] = (uint32_t)(k >> 32);
            cnt[i] = 0;
            mloc += real;
        }
        int msum = mloc;
        // block-wide sum of real entries (the list is sorted: PADs trail)
        __shared__ int red[THREADS / 32];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) msum += __shfl_xor_sync(kFull, msum, o);
        if (lane == 0) red[tid >> 5] = msum;
        __syncthreads();
        int mm = 0;
#pragma unroll
        for (int w = 0; w < THREADS / 32; w++) mm += red[w];

        if (a.mode == SVF_PRUNE_RNG) {
            const int nchunk = a.X.nchunk;
            if (stage) {
                for (int e = tid; e < mm * nchunk; e += THREADS) {
                    int i = e / nchunk, c = e % nchunk;
                    rows[e] = reinterpret_cast<const uint4 *>(row_ptr(a.X, ids[i]))[c];
                }
            }
            __syncthreads();
            const int npairs = mm * (mm - 1) / 2;
            for (int p0 = 0; p0 < npairs; p0 += nteams) {
                const int p = p0 + team;
                int i = 1, j = 0;
                const bool valid = p < npairs;
                if (valid) pair_of(p, i, j);
                const uint4 *ri, *rj;
                if (stage) {
                    ri = rows + (size_t)i * nchunk;
                    rj = rows + (size_t)j * nchunk;
                } else {
                    ri = reinterpret_cast<const uint4 *>(row_ptr(a.X, ids[i]));
                    rj = reinterpret_cast<const uint4 *>(row_ptr(a.X, ids[j]));
                }
                // invalid teams compute a harmless dummy pair (rows 0, 0)
                uint32_t key = team_pair_key<DT>(a.X.metric, valid ? rj : ri, ri, valid ? nchunk : 0, sub);
                if (valid && sub == 0 && key < dk[i]) atomicAdd(&cnt[i], 1);
            }
        } else {
            for (int e = tid; e < 2 * MAXC; e += THREADS) hkey[e] = kEmpty;
            __syncthreads();
            for (int i = tid; i < mm; i += THREADS) {
                uint32_t h = (ids[i] * 0x9E3779B1u) >> 22;  // 1024 = 2*MAXC slots
                for (int pr = 0; pr < 2 * MAXC; pr++) {
                    if (atomicCAS(&hkey[h], kEmpty, ids[i]) == kEmpty) {
                        hpos[h] = i;
                        break;
                    }
                    h = (h + 1) & (2 * MAXC - 1);
                }
            }
            __syncthreads();
            for (int e = tid; e < mm * a.nbr_w; e += THREADS) {
                const int j = e / a.nbr_w, r = e % a.nbr_w;
                const uint32_t w = __ldg(a.nbr + (int64_t)ids[j] * a.nbr_w + r);
                if (w == kEmpty) continue;
                uint32_t h = (w * 0x9E3779B1u) >> 22;
                for (int pr = 0; pr < 2 * MAXC; pr++) {
                    uint32_t kk = hkey[h];
                    if (kk == kEmpty) break;
                    if (kk == w) {
                        if (hpos[h] > j) atomicAdd(&cnt[hpos[h]], 1);
                        break;
                    }
                    h = (h + 1) & (2 * MAXC - 1);
                }
            }
        }
        __syncthreads();
        // stable sort by (count, position): the output slot of i is its rank
        uint32_t *orow = a.out_rows + li * a.R;
        for (int i = tid; i < mm; i += THREADS) {
            const int ci = cnt[i];
            int pos = 0;
            for (int j = 0; j < mm; j++) {
                const int cj = cnt[j];
                pos += (cj < ci) || (cj == ci && j < i);
            }
            if (pos < a.R) {
                orow[pos] = ids[i];
                if (a.out_dkey) a.out_dkey[li * a.R + pos] = dk[i];
            }
        }
        for (int r = mm + tid; r < a.R; r += THREADS) {
            orow[r] = kEmpty;
            if (a.out_dkey) a.out_dkey[li * a.R + r] = 0xFFFFFFFFu;
        }
        __syncthreads();
    }
}
}  // namespace

size_t prune_smem(int nchunk, bool stage) {
    size_t base = (size_t)MAXC * 4 * 3 + (size_t)2 * MAXC * 8;
    return base + (stage ? (size_t)MAXC * nchunk * 16 : 0);
}

cudaError_t launch_prune(const PruneArgs &a, int max_lists, cudaStream_t st) {
    if (a.cand_stride > MAXC) return cudaErrorInvalidValue;
    if (max_lists <= 0) return cudaSuccess;
    const int m = a.cand_stride;
    bool stage = a.mode == SVF_PRUNE_RNG && (size_t)m * a.X.nchunk * 16 <= (size_t)kPruneStageBytes;
    size_t smem = prune_smem(a.X.nchunk, false) + (stage ? (size_t)m * a.X.nchunk * 16 : 0);
    const int cap = sm_count() * 64;
    int grid = max_lists < cap ? max_lists : cap;
    if (a.X.dtype == SVF_U8) {
        cudaFuncSetAttribute(prune_kernel<SVF_U8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        prune_kernel<SVF_U8><<<grid, THREADS, smem, st>>>(a, stage ? 1 : 0);
    } else {
        cudaFuncSetAttribute(prune_kernel<SVF_F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        prune_kernel<SVF_F32><<<grid, THREADS, smem, st>>>(a, stage ? 1 : 0);
    }
    return cudaGetLastError();
}

}  // namespace svf
