// Small MLP cost model of the learned selector: in_dim -> hidden (ReLU) ->
// hidden (ReLU) -> out_dim logits, softmax cross-entropy against soft target
// distributions, trained with Adam.  All arithmetic runs in these kernels:
//   mlp_grad_kernel   : forward + backward of a chunk of samples per CTA;
//                       every gradient entry is owned by one thread, and the
//                       CTA's partial gradient is written to its own slot;
//   mlp_update_kernel : sums the CTA partials in a fixed order (deterministic)
//                       and applies one Adam step;
//   mlp_predict_kernel: forward pass and argmax (the inference kernel): one
//                       CTA per sample, weights held in registers, each
//                       layer's dot products split over all 256 threads.
// Parameter layout (row-major, one contiguous float array):
//   W1[in][h], b1[h], W2[h][h], b2[h], W3[h][out], b3[out].
#include <cmath>
#include <cstring>
#include <vector>

#include "sr_device.cuh"
#include "sr_internal.h"

namespace sr {
namespace {

constexpr int kMaxIn = 32, kMaxH = 64, kMaxOut = 64;
constexpr int kThreads = 256;
constexpr int kSamplesPerCta = 16;

struct MlpDims {
    int in, h, out;
    int64_t P;
    int64_t oW1, ob1, oW2, ob2, oW3, ob3;
};

MlpDims make_dims(int in, int h, int out) {
    MlpDims d;
    d.in = in;
    d.h = h;
    d.out = out;
    d.oW1 = 0;
    d.ob1 = d.oW1 + (int64_t)in * h;
    d.oW2 = d.ob1 + h;
    d.ob2 = d.oW2 + (int64_t)h * h;
    d.oW3 = d.ob2 + h;
    d.ob3 = d.oW3 + (int64_t)h * out;
    d.P = d.ob3 + out;
    return d;
}

// Shared-memory forward pass of one sample; returns nothing, fills h1, h2, z.
__device__ __forceinline__ void forward_one(const MlpDims& d, const float* w, const float* x, float* h1, float* h2,
                                            float* z) {
    const int t = threadIdx.x;
    if (t < d.h) {
        float a = w[d.ob1 + t];
        for (int i = 0; i < d.in; ++i) a = fmaf(x[i], w[d.oW1 + (int64_t)i * d.h + t], a);
        h1[t] = a > 0.f ? a : 0.f;
    }
    __syncthreads();
    if (t < d.h) {
        float a = w[d.ob2 + t];
        for (int j = 0; j < d.h; ++j) a = fmaf(h1[j], w[d.oW2 + (int64_t)j * d.h + t], a);
        h2[t] = a > 0.f ? a : 0.f;
    }
    __syncthreads();
    if (t < d.out) {
        float a = w[d.ob3 + t];
        for (int k = 0; k < d.h; ++k) a = fmaf(h2[k], w[d.oW3 + (int64_t)k * d.out + t], a);
        z[t] = a;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kThreads) mlp_grad_kernel(MlpDims d, const float* __restrict__ params,
                                                            const float* __restrict__ X, const float* __restrict__ Q,
                                                            int B, float* __restrict__ partial,
                                                            float* __restrict__ loss_partial) {
    extern __shared__ float sm[];
    float* w = sm;                // P
    float* g = w + d.P;           // P
    float* x = g + d.P;           // kMaxIn
    float* h1 = x + kMaxIn;       // kMaxH
    float* h2 = h1 + kMaxH;       // kMaxH
    float* z = h2 + kMaxH;        // kMaxOut
    float* dz = z + kMaxOut;      // kMaxOut
    float* dh2 = dz + kMaxOut;    // kMaxH
    float* dh1 = dh2 + kMaxH;     // kMaxH
    __shared__ float s_loss;
    const int t = threadIdx.x;
    for (int64_t i = t; i < d.P; i += blockDim.x) {
        w[i] = params[i];
        g[i] = 0.f;
    }
    if (t == 0) s_loss = 0.f;
    __syncthreads();
    const float invB = 1.0f / (float)B;
    const int b0 = blockIdx.x * kSamplesPerCta;
    const int b1 = min(B, b0 + kSamplesPerCta);
    for (int b = b0; b < b1; ++b) {
        if (t < d.in) x[t] = X[(int64_t)b * d.in + t];
        __syncthreads();
        forward_one(d, w, x, h1, h2, z);
        // softmax cross-entropy (warp 0): dz = (p - q) / B, loss += -sum q log p
        if (t < 32) {
            float m = -INFINITY;
            for (int o = t; o < d.out; o += 32) m = fmaxf(m, z[o]);
            for (int off = 16; off; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
            float s = 0.f;
            for (int o = t; o < d.out; o += 32) s += expf(z[o] - m);
            for (int off = 16; off; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            const float lse = m + logf(s);
            float l = 0.f;
            for (int o = t; o < d.out; o += 32) {
                const float q = Q[(int64_t)b * d.out + o];
                const float p = expf(z[o] - lse);
                dz[o] = (p - q) * invB;
                l += q * (lse - z[o]);
            }
            for (int off = 16; off; off >>= 1) l += __shfl_xor_sync(0xffffffffu, l, off);
            if (t == 0) s_loss += l * invB;
        }
        __syncthreads();
        // layer 3 gradients and dh2
        if (t < d.h) {
            float a = 0.f;
            for (int o = 0; o < d.out; ++o) a = fmaf(w[d.oW3 + (int64_t)t * d.out + o], dz[o], a);
            dh2[t] = h2[t] > 0.f ? a : 0.f;
        }
        for (int64_t i = t; i < (int64_t)d.h * d.out; i += blockDim.x) {
            const int k = (int)(i / d.out), o = (int)(i % d.out);
            g[d.oW3 + i] = fmaf(h2[k], dz[o], g[d.oW3 + i]);
        }
        if (t < d.out) g[d.ob3 + t] += dz[t];
        __syncthreads();
        // layer 2 gradients and dh1
        if (t < d.h) {
            float a = 0.f;
            for (int k = 0; k < d.h; ++k) a = fmaf(w[d.oW2 + (int64_t)t * d.h + k], dh2[k], a);
            dh1[t] = h1[t] > 0.f ? a : 0.f;
        }
        for (int64_t i = t; i < (int64_t)d.h * d.h; i += blockDim.x) {
            const int j = (int)(i / d.h), k = (int)(i % d.h);
            g[d.oW2 + i] = fmaf(h1[j], dh2[k], g[d.oW2 + i]);
        }
        if (t < d.h) g[d.ob2 + t] += dh2[t];
        __syncthreads();
        // layer 1 gradients
        for (int64_t i = t; i < (int64_t)d.in * d.h; i += blockDim.x) {
            const int ii = (int)(i / d.h), j = (int)(i % d.h);
            g[d.oW1 + i] = fmaf(x[ii], dh1[j], g[d.oW1 + i]);
        }
        if (t < d.h) g[d.ob1 + t] += dh1[t];
        __syncthreads();
    }
    float* out = partial + (int64_t)blockIdx.x * d.P;
    for (int64_t i = t; i < d.P; i += blockDim.x) out[i] = g[i];
    if (t == 0) loss_partial[blockIdx.x] = s_loss;
}

// Sum the per-CTA partials in CTA order, optionally export the gradient, and
// (lr > 0) apply Adam: m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
// p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
__global__ void mlp_update_kernel(int64_t P, int nparts, const float* __restrict__ partial,
                                  const float* __restrict__ loss_partial, float* __restrict__ params,
                                  float* __restrict__ m, float* __restrict__ v, float* __restrict__ grad_out,
                                  float* __restrict__ loss_out, float lr, float b1, float b2, float eps, float c1,
                                  float c2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && loss_out) {
        float l = 0.f;
        for (int k = 0; k < nparts; ++k) l += loss_partial[k];
        *loss_out = l;
    }
    if (i >= P) return;
    float gsum = 0.f;
    for (int k = 0; k < nparts; ++k) gsum += partial[(int64_t)k * P + i];
    if (grad_out) grad_out[i] = gsum;
    if (lr > 0.f) {
        const float mi = b1 * m[i] + (1.f - b1) * gsum;
        const float vi = b2 * v[i] + (1.f - b2) * gsum * gsum;
        m[i] = mi;
        v[i] = vi;
        params[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// Inference: one CTA per sample (grid-stride over the batch), 256 threads.
// Each layer's dot products are split four ways: thread (part, col) sums
// rows [part*k, part*k + k) of column col, the four partials meet in shared
// memory and are added in part order (deterministic).  Every thread loads its
// slices of W1, W2 and W3 into registers before anything waits, so the weights
// cost one trip to L2, not one per layer; the 7,400 parameters are never
// staged through shared memory.
constexpr int kParts = 4;
constexpr int kR1 = kMaxIn / kParts, kR2 = kMaxH / kParts;  // rows per part (maximum)

__global__ void __launch_bounds__(kThreads) mlp_predict_kernel(MlpDims d, const float* __restrict__ params,
                                                               const float* __restrict__ X, int B,
                                                               int* __restrict__ cls, float* __restrict__ logits) {
    __shared__ float xs[kMaxIn], h1[kMaxH], h2[kMaxH], z[kMaxOut];
    __shared__ float red[kParts][kMaxH];
    const int tid = threadIdx.x, col = tid & (kMaxH - 1), part = tid / kMaxH;
    const int k1 = (d.in + kParts - 1) / kParts, k2 = (d.h + kParts - 1) / kParts;
    // launched with programmatic stream serialisation: wait for the previous
    // kernel (a training step may have just written the parameters) before
    // any global read; only the launch latency overlaps
    grid_dependency_wait();
    allow_dependents();
    float w1[kR1], w2[kR2], w3[kR2];
#pragma unroll
    for (int r = 0; r < kR1; ++r) {
        const int j = part * k1 + r;
        w1[r] = (r < k1 && j < d.in && col < d.h) ? __ldg(params + d.oW1 + (int64_t)j * d.h + col) : 0.f;
    }
#pragma unroll
    for (int r = 0; r < kR2; ++r) {
        const int j = part * k2 + r;
        const bool row = r < k2 && j < d.h;
        w2[r] = (row && col < d.h) ? __ldg(params + d.oW2 + (int64_t)j * d.h + col) : 0.f;
        w3[r] = (row && col < d.out) ? __ldg(params + d.oW3 + (int64_t)j * d.out + col) : 0.f;
    }
    const float bias1 = (part == 0 && col < d.h) ? __ldg(params + d.ob1 + col) : 0.f;
    const float bias2 = (part == 0 && col < d.h) ? __ldg(params + d.ob2 + col) : 0.f;
    const float bias3 = (part == 0 && col < d.out) ? __ldg(params + d.ob3 + col) : 0.f;

    for (int b = blockIdx.x; b < B; b += gridDim.x) {
        if (tid < d.in) xs[tid] = X[(int64_t)b * d.in + tid];
        __syncthreads();
        float a = 0.f;
#pragma unroll
        for (int r = 0; r < kR1; ++r)
            if (r < k1 && part * k1 + r < d.in) a = fmaf(xs[part * k1 + r], w1[r], a);
        red[part][col] = a;
        __syncthreads();
        if (tid < d.h) {
            const float v = ((bias1 + red[0][tid]) + red[1][tid]) + (red[2][tid] + red[3][tid]);
            h1[tid] = v > 0.f ? v : 0.f;
        }
        __syncthreads();
        a = 0.f;
#pragma unroll
        for (int r = 0; r < kR2; ++r)
            if (r < k2 && part * k2 + r < d.h) a = fmaf(h1[part * k2 + r], w2[r], a);
        red[part][col] = a;
        __syncthreads();
        if (tid < d.h) {
            const float v = ((bias2 + red[0][tid]) + red[1][tid]) + (red[2][tid] + red[3][tid]);
            h2[tid] = v > 0.f ? v : 0.f;
        }
        __syncthreads();
        a = 0.f;
#pragma unroll
        for (int r = 0; r < kR2; ++r)
            if (r < k2 && part * k2 + r < d.h) a = fmaf(h2[part * k2 + r], w3[r], a);
        red[part][col] = a;
        __syncthreads();
        if (tid < d.out) {
            z[tid] = ((bias3 + red[0][tid]) + red[1][tid]) + (red[2][tid] + red[3][tid]);
            if (logits) logits[(int64_t)b * d.out + tid] = z[tid];
        }
        __syncthreads();
        if (tid < 32) {  // argmax, lowest index on ties
            float best = -INFINITY;
            int bi = d.out;
            for (int o = tid; o < d.out; o += 32)
                if (z[o] > best) {
                    best = z[o];
                    bi = o;
                }
            for (int off = 16; off; off >>= 1) {
                const float ob = __shfl_xor_sync(0xffffffffu, best, off);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
                if (ob > best || (ob == best && oi < bi)) {
                    best = ob;
                    bi = oi;
                }
            }
            if (tid == 0) cls[b] = bi;
        }
        // the next sample's xs write is behind the barrier after it; z and
        // red are rewritten only behind later barriers
    }
}

}  // namespace
}  // namespace sr

using namespace sr;

struct sr_mlp_s {
    MlpDims d;
    float* params = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    float* partial = nullptr;
    float* loss_partial = nullptr;
    int max_parts = 0;
    int step = 0;
};

extern "C" {

int sr_mlp_create(int in_dim, int hidden, int out_dim, sr_mlp* out) {
    if (!out || in_dim < 1 || in_dim > kMaxIn || hidden < 1 || hidden > kMaxH || out_dim < 2 || out_dim > kMaxOut)
        return SR_ERR_ARG;
    *out = nullptr;
    sr_mlp h = new sr_mlp_s;
    h->d = make_dims(in_dim, hidden, out_dim);
    const size_t pb = sizeof(float) * (size_t)h->d.P;
    cudaError_t e = cudaMalloc(&h->params, pb);
    if (e == cudaSuccess) e = cudaMalloc(&h->m, pb);
    if (e == cudaSuccess) e = cudaMalloc(&h->v, pb);
    if (e == cudaSuccess) e = cudaMemset(h->params, 0, pb);
    if (e == cudaSuccess) e = cudaMemset(h->m, 0, pb);
    if (e == cudaSuccess) e = cudaMemset(h->v, 0, pb);
    if (e != cudaSuccess) {
        sr_mlp_destroy(h);
        return status_from_cuda(e);
    }
    *out = h;
    return SR_OK;
}

int sr_mlp_destroy(sr_mlp h) {
    if (!h) return SR_OK;
    cudaFree(h->params);
    cudaFree(h->m);
    cudaFree(h->v);
    cudaFree(h->partial);
    cudaFree(h->loss_partial);
    delete h;
    return SR_OK;
}

int64_t sr_mlp_param_count(sr_mlp h) { return h ? h->d.P : -SR_ERR_ARG; }

int sr_mlp_dims(sr_mlp h, int* in_dim, int* hidden, int* out_dim) {
    if (!h || !in_dim || !hidden || !out_dim) return SR_ERR_ARG;
    *in_dim = h->d.in;
    *hidden = h->d.h;
    *out_dim = h->d.out;
    return SR_OK;
}

int sr_mlp_set_params(sr_mlp h, const float* host, int64_t count) {
    if (!h || !host || count != h->d.P) return SR_ERR_ARG;
    cudaError_t e = cudaMemcpy(h->params, host, sizeof(float) * count, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(h->m, 0, sizeof(float) * count);
    if (e == cudaSuccess) e = cudaMemset(h->v, 0, sizeof(float) * count);
    h->step = 0;
    return e == cudaSuccess ? SR_OK : status_from_cuda(e);
}

int sr_mlp_get_params(sr_mlp h, float* host, int64_t count) {
    if (!h || !host || count != h->d.P) return SR_ERR_ARG;
    cudaError_t e = cudaMemcpy(host, h->params, sizeof(float) * count, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? SR_OK : status_from_cuda(e);
}

int sr_mlp_train_step(sr_mlp h, const float* X, const float* Q, int batch, float lr, float* loss, float* grad,
                      sr_stream_t stream) {
    if (!h || !X || !Q || batch < 1 || !(lr >= 0.f)) return SR_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int parts = (batch + kSamplesPerCta - 1) / kSamplesPerCta;
    cudaError_t e;
    if (parts > h->max_parts) {
        cudaFree(h->partial);
        cudaFree(h->loss_partial);
        h->partial = nullptr;
        h->loss_partial = nullptr;
        e = cudaMalloc(&h->partial, sizeof(float) * (size_t)parts * h->d.P);
        if (e == cudaSuccess) e = cudaMalloc(&h->loss_partial, sizeof(float) * parts);
        if (e != cudaSuccess) {
            h->max_parts = 0;
            return status_from_cuda(e);
        }
        h->max_parts = parts;
    }
    const size_t smem = sizeof(float) * (size_t)(2 * h->d.P + kMaxIn + 4 * kMaxH + 2 * kMaxOut);
    int st = prepare_function((const void*)mlp_grad_kernel, smem, false);
    if (st != SR_OK) return st;
    mlp_grad_kernel<<<parts, kThreads, smem, s>>>(h->d, h->params, X, Q, batch, h->partial, h->loss_partial);
    e = cudaGetLastError();
    if (e != cudaSuccess) return status_from_cuda(e);
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    if (lr > 0.f) h->step += 1;
    const float c1 = lr > 0.f ? 1.f - powf(b1, (float)h->step) : 1.f;
    const float c2 = lr > 0.f ? 1.f - powf(b2, (float)h->step) : 1.f;
    const int blocks = (int)((h->d.P + 255) / 256);
    mlp_update_kernel<<<blocks, 256, 0, s>>>(h->d.P, parts, h->partial, h->loss_partial, h->params, h->m, h->v, grad,
                                             loss, lr, b1, b2, eps, c1, c2);
    e = cudaGetLastError();
    return e == cudaSuccess ? SR_OK : status_from_cuda(e);
}

int sr_mlp_predict(sr_mlp h, const float* X, int batch, int* cls, float* logits, sr_stream_t stream) {
    if (!h || !X || !cls || batch < 1) return SR_ERR_ARG;
    const int blocks = batch < 4096 ? batch : 4096;  // one CTA per sample, grid-stride beyond
    cudaLaunchConfig_t lc;
    std::memset(&lc, 0, sizeof lc);
    lc.gridDim = dim3(blocks);
    lc.blockDim = dim3(kThreads);
    lc.stream = (cudaStream_t)stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    const MlpDims dd = h->d;
    const float* prm = h->params;
    void* args[] = {const_cast<MlpDims*>(&dd), const_cast<float**>(&prm), const_cast<float**>(&X), &batch, &cls,
                    &logits};
    cudaError_t le = cudaLaunchKernelExC(&lc, (const void*)mlp_predict_kernel, args);
    if (le != cudaSuccess) return status_from_cuda(le);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SR_OK : status_from_cuda(e);
}

}  // extern "C"
