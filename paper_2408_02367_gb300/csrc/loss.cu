// Data-consistency residual and loss of StoDIP (Sec. 2, Eq. 2; Sec. 2.1,
// Eq. 3; Algorithm 1 line 5), summed over the coil minibatch:
//
//   r_b[j] = yhat_b[j] - y_meas[row_b][j],   L = sum_b sum_j DCF[j] |r_b[j]|^2,
//
// (||sqrt(DCF) y - sqrt(DCF) A x||^2 with a per-sample density compensation,
// DCF = 1 when none is given) and the gradient of L with respect to yhat in
// PyTorch's convention, dL/dRe + i dL/dIm = 2 DCF r, which the adjoint
// consumes in loss.backward().
//
// One pass over the residual: a block per 1024 entries of one row.  A thread
// sums its 4 entries and a warp its 128 in float32 (the FP64 pipe of this part
// is far too narrow for per-entry float64 work), the 8 warps of a block are
// added in float64 in a fixed order into one partial per block, and the last
// block to finish (device-scope counter, no waiting) sums the partials in
// float64 in a fixed order, so the loss is bitwise repeatable.
#include "sdp_internal.cuh"

namespace sdp {
namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 4;                       // residual entries per thread
constexpr int kPerBlock = kThreads * kPerThread;    // one block covers 1024 entries of one row

// Fixed-order block reduction: float32 warp butterflies, then the warps in order in float64.
__device__ __forceinline__ double block_sum_f(float v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kThreads / 32; ++w) s += red[w];
    return s;   // valid in thread 0
}

// The same in float64 throughout, for the few block partials.
__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kThreads / 32; ++w) s += red[w];
    return s;   // valid in thread 0
}

// grid = (ceil(J / 1024), B): block (x, b) handles entries [1024 x, 1024 x + 1024) of row b.
__global__ void __launch_bounds__(kThreads) residual_loss_kernel(
    const float2* yhat, const float2* __restrict__ ymeas, const int* __restrict__ meas_idx,
    const float* __restrict__ dcf, long long J, int nrows, float2* r2, double* __restrict__ partials,
    unsigned int* __restrict__ counter, float* __restrict__ loss, int* status) {
    __shared__ double red[kThreads / 32];
    __shared__ bool s_last;
    const int b = blockIdx.y;
    const int row = __ldg(meas_idx + b);
    const bool ok = row >= 0 && row < nrows;
    if (!ok && threadIdx.x == 0 && status) atomicCAS(status, 0, SDP_ERR_BOUNDS);
    const float2* h = yhat + (long long)b * J;
    const float2* m = ymeas + (long long)(ok ? row : 0) * J;
    float2* o = r2 + (long long)b * J;
    const long long j0 = (long long)blockIdx.x * kPerBlock;
    float acc = 0.f;
    // consecutive threads take consecutive entries: each pass of the block is one
    // coalesced 2 KB read of yhat and of y_meas
#pragma unroll
    for (int u = 0; u < kPerThread; ++u) {
        const long long j = j0 + u * kThreads + threadIdx.x;
        if (j < J) {
            float2 r = make_float2(0.f, 0.f);
            if (ok) {
                const float2 hv = h[j];
                const float2 mv = __ldg(m + j);
                r = make_float2(hv.x - mv.x, hv.y - mv.y);
            }
            const float wd = dcf ? __ldg(dcf + j) : 1.f;
            acc = fmaf(wd, fmaf(r.x, r.x, r.y * r.y), acc);
            o[j] = make_float2(2.f * wd * r.x, 2.f * wd * r.y);
        }
    }
    const unsigned nblk = gridDim.x * gridDim.y;
    const unsigned bid = blockIdx.y * gridDim.x + blockIdx.x;
    const double bs = block_sum_f(acc, red);
    if (threadIdx.x == 0) {
        partials[bid] = bs;
        __threadfence();
        s_last = (atomicAdd(counter, 1u) == nblk - 1);
    }
    __syncthreads();
    if (!s_last) return;
    // last block: every thread sums a fixed strided subset, then the fixed-order block sum
    __threadfence();
    double v = 0.0;
    for (unsigned i = threadIdx.x; i < nblk; i += kThreads) v += __ldcg(partials + i);
    const double tot = block_sum(v, red);
    if (threadIdx.x == 0) {
        *loss = (float)tot;
        *counter = 0u;
    }
}

}  // namespace

long long residual_loss_partials(int maxB, long long J) { return (long long)maxB * ((J + kPerBlock - 1) / kPerBlock); }

cudaError_t launch_residual_loss(const float2* yhat, const float2* ymeas, const int* meas_idx, const float* dcf, int B,
                                 long long J, int nrows, float2* r2, double* partials, unsigned int* counter,
                                 float* loss, int* status, cudaStream_t st) {
    const long long nx = (J + kPerBlock - 1) / kPerBlock;
    if (nx > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)nx, (unsigned)B);
    residual_loss_kernel<<<grid, kThreads, 0, st>>>(yhat, ymeas, meas_idx, dcf, J, nrows, r2, partials, counter,
                                                    loss, status);
    return cudaGetLastError();
}

}  // namespace sdp
