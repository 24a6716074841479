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

// Packed (Re, Im) pairs for fma.rn.f32x2: both components with one instruction,
// each rounded as a scalar fmaf would be.
__device__ __forceinline__ unsigned long long pk2(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 upk2(unsigned long long v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// The W^2 row values of one coil's window at this lane's offset (every lane
// loads: idle lanes repeat the last active lane's address and carry a zero
// coefficient).
template <int W>
__device__ __forceinline__ void row_loads(const float2* __restrict__ gb, const int (&o1)[W], const int (&o2)[W],
                                          unsigned long long (&u)[W][W]) {
#pragma unroll
    for (int a1 = 0; a1 < W; ++a1) {
        const unsigned long long* r = reinterpret_cast<const unsigned long long*>(gb + (unsigned)o1[a1]);
#pragma unroll
        for (int a2 = 0; a2 < W; ++a2) u[a1][a2] = __ldg(r + (unsigned)o2[a2]);
    }
}

// sum_{a1} phi1(a1) sum_{a2} phi2(a2) u[a1][a2], as a (Re, Im) pair.
template <int W>
__device__ __forceinline__ float2 row_sum(const unsigned long long (&w1)[W], const unsigned long long (&w2)[W],
                                          const unsigned long long (&u)[W][W]) {
    unsigned long long acc = 0ull;
#pragma unroll
    for (int a1 = 0; a1 < W; ++a1) {
        unsigned long long t = 0ull;
#pragma unroll
        for (int a2 = 0; a2 < W; ++a2) t = fma2(w2[a2], u[a1][a2], t);
        acc = fma2(w1[a1], t, acc);
    }
    return upk2(acc);
}

__device__ __forceinline__ void put(float2* __restrict__ dst, float ax, float ay, int accumulate) {
    if (accumulate) {
        const float2 old = *dst;
        ax += old.x;
        ay += old.y;
    }
    *dst = make_float2(ax, ay);
}

// Persistent CTAs of NT threads: warp w of CTA c takes the bin-sorted samples
// c (NT/32) + w + k gridDim.x (NT/32), k = 0, 1, ...: the whole grid of warps
// moves through one window of consecutive samples (their windows overlap, so
// most gathers hit L2), and the warps of a CTA, resident on one SM, take
// neighbouring samples (their gathers share the SM's L1).  NT is a plan
// choice: 1024 (the default for W <= 4: one CTA fills an SM, whose 32 warps
// take 32 consecutive samples) or 256 (more registers per thread, so more
// gathers in flight per warp).  The next sample's coordinates, frame and
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
                                                              int accumulate) {
    constexpr bool kPair = W <= 4;
    const int lane = threadIdx.x & 31;
    const long long J = g.J;
    const long long first = ((long long)blockIdx.x * NT + threadIdx.x) >> 5;
    const long long step = ((long long)gridDim.x * NT) >> 5;
    const int M1 = g.M[0], M2 = g.M[1], M3 = g.M[2];
    const long long Gk = (long long)M1 * M2 * M3 * nk;   // one coil, all channels of the call
    const int a3 = lane / cg, kg = lane - a3 * cg;
    const bool act = a3 < W;
    // idle lanes repeat the last active lane's tap and channel (an address the warp
    // reads anyway); their coefficient is zero
    const int a3c = act ? a3 : W - 1;
    const int kk = c0 + (act ? kg : cg - 1);
    const int rstride = M3 * nk;                        // one (i1, i2) row
    float4 pn = make_float4(0.f, 0.f, 0.f, 0.f);
    int tn = 0;
    float wn = 0.f;
    if (first < J) {
        pn = __ldg(pts + first);
        tn = __ldg(tframe + first);
        wn = lane < 3 * W ? __ldg(wts + first * (3 * W) + lane) : 0.f;
    }
    for (long long s = first; s < J; s += step) {
        const float4 p = pn;
        const int t = tn;
        const float wv = wn;
        const long long sn = s + step;
        if (sn < J) {
            pn = __ldg(pts + sn);
            tn = __ldg(tframe + sn);
            wn = lane < 3 * W ? __ldg(wts + sn * (3 * W) + lane) : 0.f;
        }
        const int orig = __float_as_int(p.w);
        const int m01 = (int)ceilf(p.x - g.halfW);
        const int m02 = (int)ceilf(p.y - g.halfW);
        const int m03 = (int)ceilf(p.z - g.halfW);
        // this lane's coefficient phi3(a3) V[t, kk] (0 on idle lanes) and offset within a row
        const float w3 = __shfl_sync(kFull, wv, 2 * W + a3c);
        const float2 v = act ? __ldg(V + (long long)t * g.K + k0 + kk) : make_float2(0.f, 0.f);
        const int lofs = wrap1(m03 + a3c, M3) * nk + kk;
        // row offsets (i1 M2 M3 + i2 M3) nk and the axis-1 / axis-2 weights (as (w, w)
        // pairs), the same in every lane
        unsigned long long w1[W], w2[W];
        int o1[W], o2[W];
#pragma unroll
        for (int a = 0; a < W; ++a) {
            const float v1 = __shfl_sync(kFull, wv, a);
            const float v2 = __shfl_sync(kFull, wv, W + a);
            w1[a] = pk2(v1, v1);
            w2[a] = pk2(v2, v2);
            o1[a] = wrap1(m01 + a, M1) * M2 * rstride + lofs;
            o2[a] = wrap1(m02 + a, M2) * rstride;
        }
        const float cx = w3 * v.x, cy = w3 * v.y;
        int b = 0;
        if (kPair) {
            for (; b + 1 < B; b += 2) {
                const float2* g0 = grids + (long long)b * Gk;
                unsigned long long u0[W][W], u1[W][W];
                row_loads<W>(g0, o1, o2, u0);
                row_loads<W>(g0 + Gk, o1, o2, u1);
                const float2 s0 = row_sum<W>(w1, w2, u0);
                const float2 s1 = row_sum<W>(w1, w2, u1);
                const float ax0 = cx * s0.x - cy * s0.y, ay0 = cx * s0.y + cy * s0.x;
                const float ax1 = cx * s1.x - cy * s1.y, ay1 = cx * s1.y + cy * s1.x;
                // lanes 0-15 keep coil b and send coil b + 1 to lanes 16-31, and back
                const bool hi = (lane & 16) != 0;
                float ax = hi ? ax1 : ax0, ay = hi ? ay1 : ay0;
                ax += __shfl_xor_sync(kFull, hi ? ax0 : ax1, 16);
                ay += __shfl_xor_sync(kFull, hi ? ay0 : ay1, 16);
#pragma unroll
                for (int o = 8; o > 0; o >>= 1) {
                    ax += __shfl_xor_sync(kFull, ax, o);
                    ay += __shfl_xor_sync(kFull, ay, o);
                }
                if ((lane & 15) == 0) put(y + (long long)(b + (hi ? 1 : 0)) * J + orig, ax, ay, accumulate);
            }
        }
        for (; b < B; ++b) {
            unsigned long long u[W][W];
            row_loads<W>(grids + (long long)b * Gk, o1, o2, u);
            const float2 s0 = row_sum<W>(w1, w2, u);
            float ax = cx * s0.x - cy * s0.y;
            float ay = cx * s0.y + cy * s0.x;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                ax += __shfl_xor_sync(kFull, ax, o);
                ay += __shfl_xor_sync(kFull, ay, o);
            }
            if (lane == 0) put(y + (long long)b * J + orig, ax, ay, accumulate);
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
                        const float2* grids, int B, int k0, int nk, float2* y, int accumulate, cudaStream_t st) {
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
    const long long nneed = ((long long)g.J + NT / 32 - 1) / (NT / 32);
    const unsigned nrow = (unsigned)(nneed < nres ? nneed : nres);
    constexpr int kGroup = 32 / W;   // channels per launch
    for (int c0 = 0; c0 < nk; c0 += kGroup) {
        const int cg = nk - c0 < kGroup ? nk - c0 : kGroup;
        interp_rows_kernel<W, NT><<<nrow, NT, 0, st>>>(g, pts, tframe, wts, V, grids, B, k0, nk, c0, cg, y,
                                                      accumulate || c0 > 0);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (c0 > 0) note_launches(1);   // the stage counts its first launch
    }
    return cudaSuccess;
}

template <int W>
cudaError_t launch_w(const Geo& g, int threads, const float4* pts, const int* tframe, const float* wts,
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
        return launch_rows<W, (W <= 4 ? 1024 : 256)>(g, pts, tframe, wts, V, grids, B, k0, nk, y, accumulate, st);
    return launch_rows<W, 256>(g, pts, tframe, wts, V, grids, B, k0, nk, y, accumulate, st);
}

}  // namespace

cudaError_t launch_kb_weights(const Geo& g, const float4* pts, float* wts, cudaStream_t st) {
    const long long n = (long long)g.J * 3 * g.W;
    long long nblk = (n + kThreads - 1) / kThreads;
    if (nblk > 65536) nblk = 65536;
    kb_weights_kernel<<<(unsigned)nblk, kThreads, 0, st>>>(g, pts, wts);
    return cudaGetLastError();
}

cudaError_t launch_interp(const Geo& g, int threads, const float4* pts, const int* tframe, const float* wts,
                          const float2* V, const float2* grids, int B, int k0, int nk, float2* y, int accumulate,
                          cudaStream_t st) {
    switch (g.W) {
        case 2: return launch_w<2>(g, threads, pts, tframe, wts, V, grids, B, k0, nk, y, accumulate, st);
        case 3: return launch_w<3>(g, threads, pts, tframe, wts, V, grids, B, k0, nk, y, accumulate, st);
        case 4: return launch_w<4>(g, threads, pts, tframe, wts, V, grids, B, k0, nk, y, accumulate, st);
        case 5: return launch_w<5>(g, threads, pts, tframe, wts, V, grids, B, k0, nk, y, accumulate, st);
        case 6: return launch_w<6>(g, threads, pts, tframe, wts, V, grids, B, k0, nk, y, accumulate, st);
        case 7: return launch_w<7>(g, threads, pts, tframe, wts, V, grids, B, k0, nk, y, accumulate, st);
        case 8: return launch_w<8>(g, threads, pts, tframe, wts, V, grids, B, k0, nk, y, accumulate, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sdp
