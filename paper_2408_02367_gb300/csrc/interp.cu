// Forward interpolation with the subspace contraction (gridding step A3):
//
//   y_b[j] = sum_k V[t_j, k] sum_{W^3 taps} phi(g1 - m1) phi(g2 - m2) phi(g3 - m3) U_{b,k}[m mod M]
//
// for the per-coil operator A_c of StoDIP (Sec. 2 Eq. 1, Sec. 2.1 Eq. 3): the
// temporal subspace V[t, :] is applied per sample, so the K channel grids are
// interpolated once and never expanded to T frames.  phi is the Kaiser-Bessel
// window I0(beta sqrt(1 - (2u/W)^2)) / I0(beta); the taps start at
// m0 = ceil(g - W/2), computed in float32.
//
// The 3W one-dimensional weights of every sample depend only on the
// trajectory; the plan evaluates them once (kb_weights_kernel) and both this
// kernel and the spread read them.
//
// One warp per sample (samples in bin-sorted order for locality): lanes
// 0..3W-1 load the 3W one-dimensional weights, every lane then owns
// ceil(W^3 / 32) taps whose weight and grid offset stay in registers across the
// B coils and K channels; the W taps along axis 3 are adjacent lanes reading
// adjacent addresses.  Each lane folds V[t, k] into its partial sum and a
// butterfly reduction leaves the sample value in lane 0.
#include "sdp_internal.cuh"

namespace sdp {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kThreads = 256;

__device__ __forceinline__ int wrap1(int i, int M) { return i < 0 ? i + M : (i >= M ? i - M : i); }

__global__ void kb_weights_kernel(Geo g, const float4* __restrict__ pts, float* __restrict__ wts) {
    const int W = g.W;
    const long long n = (long long)g.J * 3 * W;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const long long s = e / (3 * W);
        const int r = (int)(e - s * 3 * W);
        const int d = r / W, a = r - d * W;
        const float4 p = __ldg(pts + s);
        const float gd = d == 0 ? p.x : (d == 1 ? p.y : p.z);
        const int m0 = (int)ceilf(gd - g.halfW);
        const float u = gd - (float)(m0 + a);
        const float q = 2.f * u / (float)W;
        const float tt = fmaxf(1.f - q * q, 0.f);
        wts[e] = cyl_bessel_i0f(g.beta * sqrtf(tt)) * g.inv_i0_beta;
    }
}

template <int W, int CK>
__global__ void __launch_bounds__(kThreads) interp_kernel(Geo g, const float4* __restrict__ pts,
                                                         const int* __restrict__ tframe,
                                                         const float* __restrict__ wts,
                                                         const float2* __restrict__ V,
                                                         const float2* __restrict__ grids, int B, int k0, int nk,
                                                         float2* __restrict__ y, int accumulate) {
    constexpr int W3 = W * W * W;
    constexpr int NIT = (W3 + 31) / 32;
    const int lane = threadIdx.x & 31;
    const long long warp0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const int M1 = g.M[0], M2 = g.M[1], M3 = g.M[2];
    const long long G = (long long)M1 * M2 * M3;
    for (long long s = warp0; s < g.J; s += nwarps) {
        const float4 p = __ldg(pts + s);
        const int orig = __float_as_int(p.w);
        const int t = __ldg(tframe + s);
        const int m01 = (int)ceilf(p.x - g.halfW);
        const int m02 = (int)ceilf(p.y - g.halfW);
        const int m03 = (int)ceilf(p.z - g.halfW);
        const float wv = lane < 3 * W ? __ldg(wts + s * (3 * W) + lane) : 0.f;
        float wt[NIT];
        int off[NIT];
#pragma unroll
        for (int it = 0; it < NIT; ++it) {
            const int tau = lane + 32 * it;
            const bool valid = tau < W3;
            const int tc = valid ? tau : 0;
            const int a1 = tc / (W * W), a2 = (tc / W) % W, a3 = tc % W;
            const float w1 = __shfl_sync(kFull, wv, a1);
            const float w2 = __shfl_sync(kFull, wv, W + a2);
            const float w3 = __shfl_sync(kFull, wv, 2 * W + a3);
            wt[it] = valid ? w1 * w2 * w3 : 0.f;
            const int i1 = wrap1(m01 + a1, M1), i2 = wrap1(m02 + a2, M2), i3 = wrap1(m03 + a3, M3);
            off[it] = (i1 * M2 + i2) * M3 + i3;
        }
        const float2* Vt = V + (long long)t * g.K + k0;
        for (int b = 0; b < B; ++b) {
            float ax = 0.f, ay = 0.f;
            for (int c0 = 0; c0 < nk; c0 += CK) {
                // all CK x NIT gathers of this channel group are issued before any is used
                float2 gv[CK][NIT];
#pragma unroll
                for (int q = 0; q < CK; ++q) {
                    if (CK == 1 || c0 + q < nk) {
                        const float2* gr = grids + ((long long)b * nk + c0 + q) * G;
#pragma unroll
                        for (int it = 0; it < NIT; ++it) gv[q][it] = __ldg(gr + off[it]);
                    }
                }
#pragma unroll
                for (int q = 0; q < CK; ++q) {
                    if (CK == 1 || c0 + q < nk) {
                        float sx = 0.f, sy = 0.f;
#pragma unroll
                        for (int it = 0; it < NIT; ++it) {
                            sx = fmaf(wt[it], gv[q][it].x, sx);
                            sy = fmaf(wt[it], gv[q][it].y, sy);
                        }
                        const float2 v = __ldg(Vt + c0 + q);
                        ax += v.x * sx - v.y * sy;
                        ay += v.x * sy + v.y * sx;
                    }
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                ax += __shfl_xor_sync(kFull, ax, o);
                ay += __shfl_xor_sync(kFull, ay, o);
            }
            if (lane == 0) {
                float2* dst = y + (long long)b * g.J + orig;
                if (accumulate) {
                    const float2 old = *dst;
                    ax += old.x;
                    ay += old.y;
                }
                *dst = make_float2(ax, ay);
            }
        }
    }
}

template <int W, int CK>
cudaError_t launch_wk(const Geo& g, const float4* pts, const int* tframe, const float* wts, const float2* V,
                      const float2* grids, int B, int k0, int nk, float2* y, int accumulate, cudaStream_t st) {
    const long long warps_per_block = kThreads / 32;
    long long nblk = ((long long)g.J + warps_per_block - 1) / warps_per_block;
    if (nblk > 0x7fffffffLL) nblk = 0x7fffffffLL;
    interp_kernel<W, CK><<<(unsigned)nblk, kThreads, 0, st>>>(g, pts, tframe, wts, V, grids, B, k0, nk, y,
                                                              accumulate);
    return cudaGetLastError();
}

template <int W>
cudaError_t launch_w(const Geo& g, const float4* pts, const int* tframe, const float* wts, const float2* V,
                     const float2* grids, int B, int k0, int nk, float2* y, int accumulate, cudaStream_t st) {
    switch (channel_group(nk)) {
        case 1: return launch_wk<W, 1>(g, pts, tframe, wts, V, grids, B, k0, nk, y, accumulate, st);
        case 2: return launch_wk<W, 2>(g, pts, tframe, wts, V, grids, B, k0, nk, y, accumulate, st);
        case 3: return launch_wk<W, 3>(g, pts, tframe, wts, V, grids, B, k0, nk, y, accumulate, st);
        case 4: return launch_wk<W, 4>(g, pts, tframe, wts, V, grids, B, k0, nk, y, accumulate, st);
        case 5: return launch_wk<W, 5>(g, pts, tframe, wts, V, grids, B, k0, nk, y, accumulate, st);
        default: return launch_wk<W, 8>(g, pts, tframe, wts, V, grids, B, k0, nk, y, accumulate, st);
    }
}

}  // namespace

cudaError_t launch_kb_weights(const Geo& g, const float4* pts, float* wts, cudaStream_t st) {
    const long long n = (long long)g.J * 3 * g.W;
    long long nblk = (n + kThreads - 1) / kThreads;
    if (nblk > 65536) nblk = 65536;
    kb_weights_kernel<<<(unsigned)nblk, kThreads, 0, st>>>(g, pts, wts);
    return cudaGetLastError();
}

cudaError_t launch_interp(const Geo& g, const float4* pts, const int* tframe, const float* wts, const float2* V,
                          const float2* grids, int B, int k0, int nk, float2* y, int accumulate,
                          cudaStream_t st) {
    switch (g.W) {
        case 2: return launch_w<2>(g, pts, tframe, wts, V, grids, B, k0, nk, y, accumulate, st);
        case 3: return launch_w<3>(g, pts, tframe, wts, V, grids, B, k0, nk, y, accumulate, st);
        case 4: return launch_w<4>(g, pts, tframe, wts, V, grids, B, k0, nk, y, accumulate, st);
        case 5: return launch_w<5>(g, pts, tframe, wts, V, grids, B, k0, nk, y, accumulate, st);
        case 6: return launch_w<6>(g, pts, tframe, wts, V, grids, B, k0, nk, y, accumulate, st);
        case 7: return launch_w<7>(g, pts, tframe, wts, V, grids, B, k0, nk, y, accumulate, st);
        case 8: return launch_w<8>(g, pts, tframe, wts, V, grids, B, k0, nk, y, accumulate, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sdp
