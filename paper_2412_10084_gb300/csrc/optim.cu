// Adam update (Kingma & Ba, 2015, Algorithm 1) for the FP32 parameter
// vectors of the render (grid records, probe coefficients, MLP) and of the
// learned proposal.  One pass reads param, grad, m, v and writes param, m, v
// (and grad = 0 when asked): an HBM-streaming kernel, 16-byte vectors.
#include <cmath>

#include "internal.h"

namespace psdf {

namespace {

struct AdamArgs {
    float* p;
    float* g;
    float* m;
    float* v;
    int64_t n;
    float lr_t;   // lr * sqrt(1 - beta2^t) / (1 - beta1^t)
    float b1, b2, eps_t;  // eps * sqrt(1 - beta2^t): eps added to sqrt(v_hat)
    int clear;
};

__device__ __forceinline__ void adam1(float& p, float& g, float& m, float& v, const AdamArgs& A)
{
    m = fmaf(A.b1, m, (1.0f - A.b1) * g);
    v = fmaf(A.b2, v, (1.0f - A.b2) * g * g);
    p -= A.lr_t * m / (sqrtf(v) + A.eps_t);
    if (A.clear) g = 0.0f;
}

__global__ void adam_kernel(AdamArgs A)
{
    const int64_t n4 = A.n >> 2;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    float4* p4 = reinterpret_cast<float4*>(A.p);
    float4* g4 = reinterpret_cast<float4*>(A.g);
    float4* m4 = reinterpret_cast<float4*>(A.m);
    float4* v4 = reinterpret_cast<float4*>(A.v);
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n4; i += stride) {
        float4 p = p4[i], g = g4[i], m = m4[i], v = v4[i];
        adam1(p.x, g.x, m.x, v.x, A);
        adam1(p.y, g.y, m.y, v.y, A);
        adam1(p.z, g.z, m.z, v.z, A);
        adam1(p.w, g.w, m.w, v.w, A);
        p4[i] = p;
        m4[i] = m;
        v4[i] = v;
        if (A.clear) g4[i] = g;
    }
    // tail (n not a multiple of 4)
    const int64_t i = (n4 << 2) + int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < A.n) adam1(A.p[i], A.g[i], A.m[i], A.v[i], A);
}

}  // namespace

cudaError_t launch_adam(float* p, float* g, float* m, float* v, int64_t n, float lr, float beta1,
                        float beta2, float eps, int step, int clear_grad, cudaStream_t stream)
{
    AdamArgs A;
    A.p = p;
    A.g = g;
    A.m = m;
    A.v = v;
    A.n = n;
    const double c1 = 1.0 - std::pow(static_cast<double>(beta1), step);
    const double c2 = 1.0 - std::pow(static_cast<double>(beta2), step);
    A.lr_t = static_cast<float>(lr * std::sqrt(c2) / c1);
    A.eps_t = static_cast<float>(eps * std::sqrt(c2));
    A.b1 = beta1;
    A.b2 = beta2;
    A.clear = clear_grad;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = ((n >> 2) + 255) / 256;
    const int64_t cap = int64_t(sms > 0 ? sms : 1) * 8;
    const int blocks = static_cast<int>(want < 1 ? 1 : (want < cap ? want : cap));
    adam_kernel<<<blocks, 256, 0, stream>>>(A);
    return cudaGetLastError();
}

}  // namespace psdf
