// Spatial total-variation penalty of StoDIP (Sec. 2.1, Algorithm 1 line 6:
// loss = L_c + lambda TV(x_hat)).  The paper does not define TV; the reading
// implemented is the isotropic, epsilon-smoothed TV of every subspace channel,
// forward differences with a zero difference at the last index of each axis:
//
//   s_k(n)  = sqrt(|D1 x_k(n)|^2 + |D2 x_k(n)|^2 + |D3 x_k(n)|^2 + eps^2)
//   TV(x)   = sum_k sum_n s_k(n),      D_d x(n) = x(n + e_d) - x(n)  (0 at n_d = N_d - 1)
//   grad(m) = sum_d [ D_d x(m - e_d) / s(m - e_d) - D_d x(m) / s(m) ]
//
// grad is dTV/dRe + i dTV/dIm (PyTorch's convention).  The value is reduced
// in float64 with a fixed-order sum (bitwise repeatable); the gradient is one
// stencil pass that reads the voxel and its six neighbours (through L1).
#include "sdp_internal.cuh"

namespace sdp {
namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 4;
constexpr int kPerBlock = kThreads * kPerThread;

struct Vol {
    int N1, N2, N3;
    long long nvox;
};

__device__ __forceinline__ float2 ld(const float2* x, long long i) { return __ldg(x + i); }

// Forward differences at voxel (i1, i2, i3) of one channel (base pointer xk).
__device__ __forceinline__ void diffs(const float2* xk, const Vol& v, int i1, int i2, int i3, float2& d1, float2& d2,
                                      float2& d3) {
    const long long c = ((long long)i1 * v.N2 + i2) * v.N3 + i3;
    const float2 x0 = ld(xk, c);
    d1 = d2 = d3 = make_float2(0.f, 0.f);
    if (i1 + 1 < v.N1) {
        const float2 a = ld(xk, c + (long long)v.N2 * v.N3);
        d1 = make_float2(a.x - x0.x, a.y - x0.y);
    }
    if (i2 + 1 < v.N2) {
        const float2 a = ld(xk, c + v.N3);
        d2 = make_float2(a.x - x0.x, a.y - x0.y);
    }
    if (i3 + 1 < v.N3) {
        const float2 a = ld(xk, c + 1);
        d3 = make_float2(a.x - x0.x, a.y - x0.y);
    }
}

__device__ __forceinline__ float smag(float2 d1, float2 d2, float2 d3, float eps2) {
    return sqrtf(d1.x * d1.x + d1.y * d1.y + d2.x * d2.x + d2.y * d2.y + d3.x * d3.x + d3.y * d3.y + eps2);
}

__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kThreads / 32; ++w) s += red[w];
    return s;
}

// value: lambda * TV(x) over K channels; block b covers entries [1024 b, 1024 b + 1024)
// of the flattened [K][N1][N2][N3] array.
__global__ void __launch_bounds__(kThreads) tv_value_kernel(const float2* __restrict__ x, Vol v, long long total,
                                                           float eps, float lambda, double* __restrict__ partials,
                                                           unsigned int* __restrict__ counter, float* __restrict__ out) {
    __shared__ double red[kThreads / 32];
    __shared__ bool s_last;
    const float eps2 = eps * eps;
    double acc = 0.0;
#pragma unroll
    for (int u = 0; u < kPerThread; ++u) {
        const long long e = (long long)blockIdx.x * kPerBlock + u * kThreads + threadIdx.x;
        if (e < total) {
            const long long k = e / v.nvox;
            const long long r = e - k * v.nvox;
            const int i3 = (int)(r % v.N3);
            const long long r12 = r / v.N3;
            const int i2 = (int)(r12 % v.N2), i1 = (int)(r12 / v.N2);
            float2 d1, d2, d3;
            diffs(x + k * v.nvox, v, i1, i2, i3, d1, d2, d3);
            acc += (double)smag(d1, d2, d3, eps2);
        }
    }
    const double bs = block_sum(acc, red);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = bs;
        __threadfence();
        s_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double t = 0.0;
    for (unsigned i = threadIdx.x; i < gridDim.x; i += kThreads) t += __ldcg(partials + i);
    const double tot = block_sum(t, red);
    if (threadIdx.x == 0) {
        *out = (float)((double)lambda * tot);
        *counter = 0u;
    }
}

// gradient: out = (accumulate ? out : 0) + lambda * (*scale) * grad TV
__global__ void __launch_bounds__(kThreads) tv_grad_kernel(const float2* __restrict__ x, Vol v, long long total,
                                                          float eps, float lambda, const float* __restrict__ scale,
                                                          float2* __restrict__ out, int accumulate) {
    const float eps2 = eps * eps;
    const float f = lambda * (scale ? __ldg(scale) : 1.f);
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long k = e / v.nvox;
        const long long r = e - k * v.nvox;
        const int i3 = (int)(r % v.N3);
        const long long r12 = r / v.N3;
        const int i2 = (int)(r12 % v.N2), i1 = (int)(r12 / v.N2);
        const float2* xk = x + k * v.nvox;
        float2 d1, d2, d3;
        diffs(xk, v, i1, i2, i3, d1, d2, d3);
        const float is0 = 1.f / smag(d1, d2, d3, eps2);
        float gx = -(d1.x + d2.x + d3.x) * is0, gy = -(d1.y + d2.y + d3.y) * is0;
        float2 b1, b2, b3;
        if (i1 > 0) {
            diffs(xk, v, i1 - 1, i2, i3, b1, b2, b3);
            const float is = 1.f / smag(b1, b2, b3, eps2);
            gx += b1.x * is;
            gy += b1.y * is;
        }
        if (i2 > 0) {
            diffs(xk, v, i1, i2 - 1, i3, b1, b2, b3);
            const float is = 1.f / smag(b1, b2, b3, eps2);
            gx += b2.x * is;
            gy += b2.y * is;
        }
        if (i3 > 0) {
            diffs(xk, v, i1, i2, i3 - 1, b1, b2, b3);
            const float is = 1.f / smag(b1, b2, b3, eps2);
            gx += b3.x * is;
            gy += b3.y * is;
        }
        float2 g = make_float2(f * gx, f * gy);
        if (accumulate) {
            const float2 o = out[e];
            g.x += o.x;
            g.y += o.y;
        }
        out[e] = g;
    }
}

}  // namespace

long long tv_partials(int K, long long nvox) { return ((long long)K * nvox + kPerBlock - 1) / kPerBlock; }

cudaError_t launch_tv_value(const Geo& g, const float2* x, float eps, float lambda, double* partials,
                            unsigned int* counter, float* out, cudaStream_t st) {
    Vol v{g.N[0], g.N[1], g.N[2], (long long)g.N[0] * g.N[1] * g.N[2]};
    const long long total = (long long)g.K * v.nvox;
    const long long nblk = (total + kPerBlock - 1) / kPerBlock;
    if (nblk > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    tv_value_kernel<<<(unsigned)nblk, kThreads, 0, st>>>(x, v, total, eps, lambda, partials, counter, out);
    return cudaGetLastError();
}

cudaError_t launch_tv_grad(const Geo& g, const float2* x, float eps, float lambda, const float* scale, float2* out,
                           int accumulate, cudaStream_t st) {
    Vol v{g.N[0], g.N[1], g.N[2], (long long)g.N[0] * g.N[1] * g.N[2]};
    const long long total = (long long)g.K * v.nvox;
    long long nblk = (total + kThreads - 1) / kThreads;
    if (nblk > 65535LL * 16) nblk = 65535LL * 16;
    tv_grad_kernel<<<(unsigned)nblk, kThreads, 0, st>>>(x, v, total, eps, lambda, scale, out, accumulate);
    return cudaGetLastError();
}

}  // namespace sdp
