// svf_update.h -- launchers of the insert / delete / codec kernels (update.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "svf_dev.cuh"

namespace svf {

constexpr int kMaxRepair = 512;  // candidates of one localized repair (c * R)

// An update that runs while searches of the previous epoch may still be
// reading the graph (the serving loop's update stream): before any kernel
// rewrites an existing row, the row is copied into this update's half of the
// shadow rows and stamped row_ver = E; a deleted vertex gets del_ep = E
// before its bit is set (see VerCtx for the reading side).
struct VerUpd {
    uint32_t E;                    // the update's number (>= 1)
    uint32_t *row_ver;             // [n_cap]
    int32_t *shadow_slot;          // [n_cap]
    uint32_t *shadow;              // all shadow rows [2 cap][R]
    int64_t base;                  // first row of this update's half (0 or cap)
    int64_t cap;                   // rows per half
    uint32_t *del_ep;              // [n_cap]
    unsigned long long *counter;   // rows shadowed by this update (zeroed before it)
};

// Reverse edges of the new rows n0 .. n0+m-1 into the tail halves of their
// targets; targets >= tmax are skipped (an insert passes tmax = n0).
cudaError_t launch_reverse_patch(const RowDesc &X, uint32_t *graph, int R, const uint32_t *del, int64_t n0, int64_t m,
                                 const uint32_t *rows, const uint32_t *dkeys, int64_t tmax, int32_t *head,
                                 int32_t *next, unsigned long long *status, cudaStream_t st,
                                 const VerUpd *ver = nullptr);
cudaError_t launch_iota(uint32_t *out, int64_t m, int64_t base, cudaStream_t st);
cudaError_t launch_delete_mark(const uint32_t *ids, int64_t m, int64_t n_used, uint32_t *del,
                               unsigned long long *status, cudaStream_t st, const VerUpd *ver = nullptr);
// Shadow and stamp the rows vl[0..nv) before they are rewritten.
cudaError_t launch_stamp_rows(const uint32_t *graph, int R, const uint32_t *vl, int64_t nv, const VerUpd &ver,
                              unsigned long long *status, cudaStream_t st);
cudaError_t launch_delete_scan(const uint32_t *graph, int R, const uint32_t *del, int64_t n_used, int min_del,
                               uint32_t *vl, unsigned long long *status, cudaStream_t st);
cudaError_t launch_delete_gather(const RowDesc &X, const uint32_t *graph, int R, const uint32_t *del, int64_t n_used,
                                 int c, int cap, const uint32_t *vl, int64_t v0, int64_t nv, uint64_t *cand,
                                 int cstride, cudaStream_t st);
cudaError_t launch_delete_finalize(uint32_t *graph, int R, const uint32_t *del, const uint32_t *vl, int64_t nv,
                                   const uint32_t *newrows, cudaStream_t st);

}  // namespace svf
