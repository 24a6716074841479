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
// One warp per sample (samples in bin-sorted order for locality).  The grids
// are channel-interleaved, [b][i1][i2][i3][kk], so the W taps along axis 3 of
// one (i1, i2) row of the window, for all nk channels, are one contiguous run
// of W nk values.
//
// Row kernel (nk >= 2): lane l owns the axis-3 tap a3 = l / cg and the channel
// kk = c0 + l % cg of a group of cg <= 32 / W channels (lanes beyond W cg
// idle).  Its coefficient phi3(a3) V[t, kk] and its offset within a row are
// fixed for the sample; for each coil the warp then walks the W^2 rows of the
// window, one load per lane and row (the warp reads one contiguous run per
// row), weights them by phi1 phi2 (the same in every lane), multiplies by the
// lane's coefficient and reduces over the warp.  More than 32 / W channels run
// as several launches, each adding its group's sum into y.
//
// Tap kernel (nk == 1): lanes own ceil(W^3 / 32) taps each, whose weights and
// offsets stay in registers across the coils; the W taps of a row are adjacent
// lanes reading adjacent addresses.
#include <atomic>

#include "interp_impl.cuh"

namespace sdp {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kThreads = 256;

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

// Persistent CTAs of NT threads: warp w of CTA c takes the bin-sorted samples
// c (NT/32) + w + k gridDim.x (NT/32), k = 0, 1, ...: the whole grid of warps
// moves through one window of consecutive samples (their windows overlap, so
// most gathers hit L2), and the warps of a CTA, resident on one SM, take
// neighbouring samples (their gathers share the SM's L1).  NT is a plan
// choice: 256 (the default) or 1024 (W <= 4: one CTA fills an SM, whose 32
// warps take 32 consecutive samples; on par for one or two coils, far slower
// for eight, whose windows no longer fit the SM's L1 together).  The next sample's coordinates, frame and
// weights are loaded while the current one is interpolated.  For W <= 4 the gathers of two coils are issued together and
// the two sums share one warp reduction (lanes 0-15 finish coil b, lanes
// 16-31 coil b + 1).
template <int W, int NT>
__global__ void __launch_bounds__(NT) interp_rows_kernel(Geo g, const float4* __restrict__ pts,
                                                              const int* __restrict__ tframe,
                                                              const float* __restrict__ wts,
                                                              const float2* __restrict__ V,
                                                              const float2* __restrict__ grids, int B, int k0,
                                                              int nk, int c0, int cg, float2* __restrict__ y,
                                                              int accumulate, int run, int cblock) {
    const int lane = threadIdx.x & 31;
    const long long J = g.J;
    const long long first = ((long long)blockIdx.x * NT + threadIdx.x) >> 5;
    const long long step = ((long long)gridDim.x * NT) >> 5;
    const RowLane rl = row_lane<W>(lane, c0, cg);
    const long long Gk = (long long)g.M[0] * g.M[1] * g.M[2] * nk;
    // the samples are swept once per block of cblock coils (all B coils when cblock = 0):
    // a sweep's gathers then touch only that block's grids
    const int cb = cblock > 0 && cblock < B ? cblock : B;
    for (int b0 = 0; b0 < B; b0 += cb) {
    const int nb = min(cb, B - b0);
    float4 pn = make_float4(0.f, 0.f, 0.f, 0.f);
    int tn = 0;
    float wn = 0.f;
    long long s = first * run;    // warp w takes the runs w, w + step, ... of `run` consecutive samples
    int r = 0;
    if (s < J) {
        pn = __ldg(pts + s);
        tn = __ldg(tframe + s);
        wn = lane < 3 * W ? __ldg(wts + s * (3 * W) + lane) : 0.f;
    }
    while (s < J) {
        const float4 p = pn;
        const int t = tn;
        const float wv = wn;
        const bool in_run = r + 1 < run;
        const long long sn = in_run ? s + 1 : s - r + step * run;
        r = in_run ? r + 1 : 0;
        if (sn < J) {
            pn = __ldg(pts + sn);
            tn = __ldg(tframe + sn);
            wn = lane < 3 * W ? __ldg(wts + sn * (3 * W) + lane) : 0.f;
        }
        interp_rows_sample<W>(g, rl, V, grids + b0 * Gk, nb, k0, nk, y + b0 * J, accumulate, p, t, wv, lane);
        s = sn;
    }
    }
}

template <int W>
__global__ void __launch_bounds__(kThreads) interp_taps_kernel(Geo g, const float4* __restrict__ pts,
                                                              const int* __restrict__ tframe,
                                                              const float* __restrict__ wts,
                                                              const float2* __restrict__ V,
                                                              const float2* __restrict__ grids, int B, int k0,
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
        const float2 v = __ldg(V + (long long)t * g.K + k0);
        for (int b = 0; b < B; ++b) {
            const float2* gr = grids + (long long)b * G;
            float2 gv[NIT];
#pragma unroll
            for (int it = 0; it < NIT; ++it) gv[it] = __ldg(gr + off[it]);
            float sx = 0.f, sy = 0.f;
#pragma unroll
            for (int it = 0; it < NIT; ++it) {
                sx = fmaf(wt[it], gv[it].x, sx);
                sy = fmaf(wt[it], gv[it].y, sy);
            }
            float ax = v.x * sx - v.y * sy;
            float ay = v.x * sy + v.y * sx;
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

template <int W, int NT>
cudaError_t launch_rows(const Geo& g, const float4* pts, const int* tframe, const float* wts, const float2* V,
                        const float2* grids, int B, int k0, int nk, float2* y, int accumulate, int run,
                        int cblock, cudaStream_t st) {
    // persistent grid: the CTAs that are resident at once (or fewer for a short trajectory)
    static std::atomic<int> resident{0};
    int per_sm = resident.load(std::memory_order_relaxed);
    if (per_sm == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, interp_rows_kernel<W, NT>, NT, 0) !=
                cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        resident.store(per_sm, std::memory_order_relaxed);
    }
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess || nsm < 1)
        return cudaErrorInvalidDevice;
    const long long nres = (long long)nsm * per_sm;
    const long long nneed = ((long long)g.J + (long long)run * (NT / 32) - 1) / ((long long)run * (NT / 32));
    const unsigned nrow = (unsigned)(nneed < nres ? nneed : nres);
    constexpr int kGroup = 32 / W;   // channels per launch
    for (int c0 = 0; c0 < nk; c0 += kGroup) {
        const int cg = nk - c0 < kGroup ? nk - c0 : kGroup;
        interp_rows_kernel<W, NT><<<nrow, NT, 0, st>>>(g, pts, tframe, wts, V, grids, B, k0, nk, c0, cg, y,
                                                      accumulate || c0 > 0, run, cblock);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (c0 > 0) note_launches(1);   // the stage counts its first launch
    }
    return cudaSuccess;
}

template <int W>
cudaError_t launch_w(const Geo& g, int threads, int run, int cblock, const float4* pts, const int* tframe,
                     const float* wts,
                     const float2* V, const float2* grids, int B, int k0, int nk, float2* y, int accumulate,
                     cudaStream_t st) {
    if (nk == 1) {
        const long long warps_per_block = kThreads / 32;
        long long nblk = ((long long)g.J + warps_per_block - 1) / warps_per_block;
        if (nblk > 0x7fffffffLL) nblk = 0x7fffffffLL;
        interp_taps_kernel<W><<<(unsigned)nblk, kThreads, 0, st>>>(g, pts, tframe, wts, V, grids, B, k0, y,
                                                                  accumulate);
        return cudaGetLastError();
    }
    if (W <= 4 && threads == 1024)
        return launch_rows<W, (W <= 4 ? 1024 : 256)>(g, pts, tframe, wts, V, grids, B, k0, nk, y, accumulate, run,
                                                     cblock, st);
    return launch_rows<W, 256>(g, pts, tframe, wts, V, grids, B, k0, nk, y, accumulate, run, cblock, st);
}

}  // namespace

cudaError_t launch_kb_weights(const Geo& g, const float4* pts, float* wts, cudaStream_t st) {
    const long long n = (long long)g.J * 3 * g.W;
    long long nblk = (n + kThreads - 1) / kThreads;
    if (nblk > 65536) nblk = 65536;
    kb_weights_kernel<<<(unsigned)nblk, kThreads, 0, st>>>(g, pts, wts);
    return cudaGetLastError();
}

cudaError_t launch_interp(const Geo& g, int threads, int run, int cblock, const float4* pts, const int* tframe,
                          const float* wts,
                          const float2* V, const float2* grids, int B, int k0, int nk, float2* y, int accumulate,
                          cudaStream_t st) {
    if (run < 1) run = 1;
    switch (g.W) {
        case 2: return launch_w<2>(g, threads, run, cblock, pts, tframe, wts, V, grids, B, k0, nk, y, accumulate, st);
        case 3: return launch_w<3>(g, threads, run, cblock, pts, tframe, wts, V, grids, B, k0, nk, y, accumulate, st);
        case 4: return launch_w<4>(g, threads, run, cblock, pts, tframe, wts, V, grids, B, k0, nk, y, accumulate, st);
        case 5: return launch_w<5>(g, threads, run, cblock, pts, tframe, wts, V, grids, B, k0, nk, y, accumulate, st);
        case 6: return launch_w<6>(g, threads, run, cblock, pts, tframe, wts, V, grids, B, k0, nk, y, accumulate, st);
        case 7: return launch_w<7>(g, threads, run, cblock, pts, tframe, wts, V, grids, B, k0, nk, y, accumulate, st);
        case 8: return launch_w<8>(g, threads, run, cblock, pts, tframe, wts, V, grids, B, k0, nk, y, accumulate, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sdp
