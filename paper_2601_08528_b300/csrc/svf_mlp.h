// svf_mlp.h -- sizes and launchers of the stop-network kernels (mlp.cu).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace svf {

constexpr int kMlpIn = 16, kMlpHidden = 64;
constexpr int kMlpParams = kMlpHidden * kMlpIn + 2 * kMlpHidden + 1;  // 1153
constexpr int kMlpParams1 = kMlpParams + 1;                           // + the loss slot
constexpr int kMlpPacked = 1160;                                      // bf16 entries (padded)
constexpr int kMlpOffB1 = kMlpHidden * kMlpIn, kMlpOffW2 = kMlpOffB1 + kMlpHidden, kMlpOffB2 = kMlpOffW2 + kMlpHidden;

size_t mlp_grad_partial_floats(int64_t B);
cudaError_t launch_mlp_grad(const float *feat, const int32_t *meta, int T, const int32_t *idx, int64_t B,
                            const float *prm, float *grad, float *partial, float *loss, cudaStream_t st);
cudaError_t launch_mlp_adam(float *prm, const float *grad, float *m, float *v, int64_t step, float lr, float b1,
                            float b2, float eps, cudaStream_t st);
cudaError_t launch_mlp_pack(const float *prm, void *packed, cudaStream_t st);
cudaError_t launch_mlp_forward(const float *prm, const float *feat, int64_t n, float *z, cudaStream_t st);

}  // namespace svf
