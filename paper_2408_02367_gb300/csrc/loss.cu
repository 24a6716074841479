// Data-consistency residual and loss of StoDIP (Sec. 2.1, Eq. 3 with DCF = 1,
// Algorithm 1 line 5), summed over the coil minibatch:
//
//   r_b[j] = yhat_b[j] - y_meas[row_b][j],   L = sum_b sum_j |r_b[j]|^2,
//
// and the gradient of L with respect to yhat in PyTorch's convention,
// dL/dRe + i dL/dIm = 2 r, which the adjoint consumes in loss.backward().
//
// One pass over the residual: every thread accumulates |r|^2 in float64,
// blocks reduce in shared memory and write one partial each; the last block
// to finish (device-scope counter, no waiting) sums the partials in block
// order, so the loss is bitwise repeatable.
#include "sdp_internal.cuh"

namespace sdp {
namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) residual_loss_kernel(
    const float2* yhat, const float2* __restrict__ ymeas, const int* __restrict__ meas_idx,
    int B, long long J, int nrows, float2* r2, double* __restrict__ partials,
    unsigned int* __restrict__ counter, float* __restrict__ loss, int* status) {
    __shared__ double red[kThreads / 32];
    __shared__ bool s_last;
    double acc = 0.0;
    const long long total = (long long)B * J;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(e / J);
        const long long j = e - (long long)b * J;
        const int row = __ldg(meas_idx + b);
        float2 r;
        if (row >= 0 && row < nrows) {
            const float2 h = yhat[e];
            const float2 m = __ldg(ymeas + (long long)row * J + j);
            r = make_float2(h.x - m.x, h.y - m.y);
        } else {
            if (status) atomicCAS(status, 0, SDP_ERR_BOUNDS);
            r = make_float2(0.f, 0.f);
        }
        acc += (double)r.x * r.x + (double)r.y * r.y;
        r2[e] = make_float2(2.f * r.x, 2.f * r.y);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += red[w];
        partials[blockIdx.x] = s;
        __threadfence();
        const unsigned prev = atomicAdd(counter, 1u);
        s_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        double s = 0.0;
        for (unsigned i = 0; i < gridDim.x; ++i) s += __ldcg(partials + i);
        *loss = (float)s;
        *counter = 0u;
    }
}

}  // namespace

int residual_loss_blocks() { return 2 * 152; }

cudaError_t launch_residual_loss(const float2* yhat, const float2* ymeas, const int* meas_idx, int B, long long J,
                                 int nrows, float2* r2, double* partials, unsigned int* counter, float* loss,
                                 int* status, cudaStream_t st) {
    residual_loss_kernel<<<residual_loss_blocks(), kThreads, 0, st>>>(yhat, ymeas, meas_idx, B, J, nrows, r2,
                                                                     partials, counter, loss, status);
    return cudaGetLastError();
}

}  // namespace sdp
