// mlp.cu -- training and packing of the learned early-stop network
// (16 features -> 64 ReLU -> 1 logit; the search stops once the logit
// reaches logit(tau)).  Samples are the per-iteration rows of a search trace
// ([nq][T][16] features + per-query (iterations run, last top-k change));
// the label of iteration t of query q is t >= t_last(q), i.e. "the top-k set
// has already reached its final value".
//
// Loss: mean binary cross-entropy over a minibatch.  Gradients are reduced
// in a fixed order (per-block partial sums, then a sum over blocks), so
// training is deterministic.  Parameter vector layout (fp32 master, and the
// packed bf16 copy the search kernel reads): W1[64][16], b1[64], w2[64], b2.
#include <cstdint>

#include "svf_internal.h"
#include "svf_mlp.h"

namespace svf {

namespace {
constexpr int NF = kMlpIn, NH = kMlpHidden;
constexpr int BS = 256;  // samples per block

__device__ __forceinline__ float softplus(float z) { return z > 0.f ? z + log1pf(expf(-z)) : log1pf(expf(z)); }

__global__ void __launch_bounds__(BS) mlp_grad_kernel(const float *feat, const int32_t *meta, int T, const int32_t *idx,
                                                      int64_t B, const float *prm, float *partial) {
    extern __shared__ __align__(16) float sh[];
    float *sf = sh;              // [BS][NF]
    float *sd = sf + BS * NF;    // [BS][NH] dL/dh (masked)
    float *sa = sd + BS * NH;    // [BS][NH] relu(h)
    float *sz = sa + BS * NH;    // [BS] dL/dz
    float *sl = sz + BS;         // [BS] loss terms
    const int tid = threadIdx.x;
    const int64_t s = (int64_t)blockIdx.x * BS + tid;
    const float *W1 = prm, *b1 = prm + NH * NF, *w2 = b1 + NH, b2 = w2[NH];
    float f[NF];
    float dz = 0.f, lt = 0.f;
    const bool valid = s < B;
    if (valid) {
        const int32_t id = idx[s];
        const int q = id / T, t = id % T;
        const float y = (t >= meta[2 * q + 1]) ? 1.f : 0.f;
#pragma unroll
        for (int i = 0; i < NF; i++) f[i] = feat[(int64_t)id * NF + i];
        float z = b2;
        for (int j = 0; j < NH; j++) {
            float h = b1[j];
#pragma unroll
            for (int i = 0; i < NF; i++) h = fmaf(W1[j * NF + i], f[i], h);
            const float a = h > 0.f ? h : 0.f;
            sa[tid * NH + j] = a;
            z = fmaf(w2[j], a, z);
        }
        const float p = 1.f / (1.f + expf(-z));
        dz = (p - y) / (float)B;
        lt = softplus(z) - y * z;
        for (int j = 0; j < NH; j++) sd[tid * NH + j] = sa[tid * NH + j] > 0.f ? dz * w2[j] : 0.f;
    } else {
#pragma unroll
        for (int i = 0; i < NF; i++) f[i] = 0.f;
        for (int j = 0; j < NH; j++) {
            sa[tid * NH + j] = 0.f;
            sd[tid * NH + j] = 0.f;
        }
    }
#pragma unroll
    for (int i = 0; i < NF; i++) sf[tid * NF + i] = f[i];
    sz[tid] = dz;
    sl[tid] = lt;
    __syncthreads();
    // gradient entries, each a sum over the block's samples in sample order
    float *out = partial + (int64_t)blockIdx.x * kMlpParams1;
    for (int e = tid; e < kMlpParams1; e += BS) {
        float acc = 0.f;
        if (e < NH * NF) {
            const int j = e / NF, i = e % NF;
            for (int r = 0; r < BS; r++) acc = fmaf(sd[r * NH + j], sf[r * NF + i], acc);
        } else if (e < NH * NF + NH) {
            const int j = e - NH * NF;
            for (int r = 0; r < BS; r++) acc += sd[r * NH + j];
        } else if (e < NH * NF + 2 * NH) {
            const int j = e - NH * NF - NH;
            for (int r = 0; r < BS; r++) acc = fmaf(sa[r * NH + j], sz[r], acc);
        } else if (e == kMlpParams) {
            for (int r = 0; r < BS; r++) acc += sz[r];
            out[kMlpParams - 1] = acc;  // b2
            acc = 0.f;
            for (int r = 0; r < BS; r++) acc += sl[r];
        }
        if (e < kMlpParams - 1) out[e] = acc;
        else if (e == kMlpParams) out[kMlpParams] = acc;  // loss sum
    }
}

__global__ void mlp_reduce_kernel(const float *partial, int nblk, int64_t B, float *grad, float *loss) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e > kMlpParams) return;
    float acc = 0.f;
    for (int b = 0; b < nblk; b++) acc += partial[(int64_t)b * kMlpParams1 + e];
    if (e < kMlpParams) grad[e] = acc;
    else if (loss) *loss = acc / (float)B;
}

__global__ void mlp_adam_kernel(float *prm, const float *grad, float *m, float *v, float lr, float b1, float b2,
                                float eps, float c1, float c2) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kMlpParams) return;
    const float g = grad[e];
    const float mm = b1 * m[e] + (1.f - b1) * g;
    const float vv = b2 * v[e] + (1.f - b2) * g * g;
    m[e] = mm;
    v[e] = vv;
    prm[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

__global__ void mlp_pack_kernel(const float *prm, __nv_bfloat16 *out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < kMlpParams) out[e] = __float2bfloat16_rn(prm[e]);
    else if (e < kMlpPacked) out[e] = __float2bfloat16_rn(0.f);
}

// logits of the fp32 network (the training forward), one thread per sample
__global__ void mlp_forward_kernel(const float *prm, const float *feat, int64_t n, float *z) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const float *W1 = prm, *b1 = prm + NH * NF, *w2 = b1 + NH;
    float f[NF];
#pragma unroll
    for (int i = 0; i < NF; i++) f[i] = feat[s * NF + i];
    float acc = w2[NH];
    for (int j = 0; j < NH; j++) {
        float h = b1[j];
#pragma unroll
        for (int i = 0; i < NF; i++) h = fmaf(W1[j * NF + i], f[i], h);
        if (h > 0.f) acc = fmaf(w2[j], h, acc);
    }
    z[s] = acc;
}
}  // namespace

size_t mlp_grad_partial_floats(int64_t B) { return (size_t)((B + BS - 1) / BS) * kMlpParams1; }

cudaError_t launch_mlp_grad(const float *feat, const int32_t *meta, int T, const int32_t *idx, int64_t B,
                            const float *prm, float *grad, float *partial, float *loss, cudaStream_t st) {
    const int nblk = (int)((B + BS - 1) / BS);
    const size_t smem = sizeof(float) * (BS * NF + 2 * BS * NH + 2 * BS);
    cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    mlp_grad_kernel<<<nblk, BS, smem, st>>>(feat, meta, T, idx, B, prm, partial);
    mlp_reduce_kernel<<<(kMlpParams + 1 + 127) / 128, 128, 0, st>>>(partial, nblk, B, grad, loss);
    return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float *prm, const float *grad, float *m, float *v, int64_t step, float lr, float b1,
                            float b2, float eps, cudaStream_t st) {
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    mlp_adam_kernel<<<(kMlpParams + 127) / 128, 128, 0, st>>>(prm, grad, m, v, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t launch_mlp_pack(const float *prm, void *packed, cudaStream_t st) {
    mlp_pack_kernel<<<(kMlpPacked + 127) / 128, 128, 0, st>>>(prm, reinterpret_cast<__nv_bfloat16 *>(packed));
    return cudaGetLastError();
}

cudaError_t launch_mlp_forward(const float *prm, const float *feat, int64_t n, float *z, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    mlp_forward_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(prm, feat, n, z);
    return cudaGetLastError();
}

}  // namespace svf
