// Forward interpolation building blocks (included by interp.cu and batch.cu):
// packed (Re, Im) arithmetic, the W^2 row gathers of one window and the whole
// step A3 for one bin-sorted sample of one plan,
//
//   y_b[j] = sum_k V[t_j, k] sum_{W^3 taps} phi(g1 - m1) phi(g2 - m2) phi(g3 - m3) U_{b,k}[m mod M],
//
// on channel-interleaved grids [b][i1][i2][i3][kk] (see interp.cu for the
// lane layout).  interp.cu runs it over one plan's samples, batch.cu over the
// samples of several plans in one launch.
#pragma once

#include "index_map.cuh"
#include "sdp_internal.cuh"

namespace sdp {
namespace {

constexpr unsigned kFullI = 0xffffffffu;

__device__ __forceinline__ int wrap1(int i, int M) { return i < 0 ? i + M : (i >= M ? i - M : i); }

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

// The lane's fixed role in the row kernel: axis-3 tap a3c and channel kk of a
// group of cg <= 32 / W channels starting at c0 (idle lanes, a3 >= W, repeat
// the last active lane's tap and channel with a zero coefficient).
using RowLane = imap::RowLane;

template <int W>
__device__ __forceinline__ RowLane row_lane(int lane, int c0, int cg) {
    return imap::row_lane_map(lane, c0, cg, W);
}

// Step A3 for one sample (grid coordinates and original index p, frame t, this
// lane's entry wv of the sample's 3W plan-time weights) and every coil b < B:
// y[b][orig] (+)= sum over the group's channels.  For W <= 4 the gathers of
// two coils are issued together and the two sums share one warp reduction
// (lanes 0-15 finish coil b, lanes 16-31 coil b + 1).
template <int W>
__device__ __forceinline__ void interp_rows_sample(const Geo& g, const RowLane& rl, const float2* __restrict__ V,
                                                   const float2* __restrict__ grids, int B, int k0, int nk,
                                                   float2* __restrict__ y, int accumulate, float4 p, int t, float wv,
                                                   int lane) {
    constexpr bool kPair = W <= 4;
    constexpr unsigned kFull = kFullI;
    const long long J = g.J;
    const int M1 = g.M[0], M2 = g.M[1], M3 = g.M[2];
    const long long Gk = (long long)M1 * M2 * M3 * nk;   // one coil, all channels of the call
    const int a3c = rl.a3c, kk = rl.kk;
    const bool act = rl.act;
    const int rstride = M3 * nk;                        // one (i1, i2) row
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

}  // namespace
}  // namespace sdp
