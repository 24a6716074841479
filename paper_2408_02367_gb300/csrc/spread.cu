// Adjoint spreading with the conjugate subspace weights (gridding step A5):
//
//   H_{b,k}[m mod M] = sum_j phi(g_j1 - m1) phi(g_j2 - m2) phi(g_j3 - m3) conj(V[t_j, k]) r_b[j]
//
// the first step of A_c^H, which Algorithm 1 of StoDIP needs for
// loss.backward() (Sec. 2.1, Eq. 3).  conj(V[t_j, k]) r_b[j] folds the
// temporal subspace into the spread, so only K channel grids are formed.
//
// Owner-computes bins.  The grid is cut into bins of bs1 x bs2 x bs3 points.
// The plan lists, per bin, every sample whose W^3 window touches the bin (the
// incidences), split into chunks of bounded length (the subproblems).  A CTA
// takes one subproblem for one coil b: it accumulates the taps that fall
// inside its bin into a shared-memory tile (all K channels) with shared
// atomics, a warp per incidence and lanes over taps, then
//   - single-chunk bin: stores the tile straight into the grid;
//   - multi-chunk bin (the dense k-space centre): stores its partial tile,
//     and the last chunk to finish (device-scope counter, no waiting) sums all
//     partials in chunk order and stores the bin.
// Every grid point is written exactly once by plain stores: no zero fill of
// the grid and no global atomics on it.
#include "sdp_internal.cuh"

namespace sdp {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kThreads = 256;

__device__ __forceinline__ int wrap1(int i, int M) { return i < 0 ? i + M : (i >= M ? i - M : i); }

struct SpreadArgs {
    Geo g;
    int bs1, bs2, bs3;
    int nb1, nb2, nb3;
    const SubProb* subs;
    const int* inc;
    const float4* pts;
    const int* tframe;
    const float2* V;
    const float2* y;
    const float* scale;
    int k0, nk;
    float2* grids;
    float2* partials;
    long long slots_per_b;
    long long slot_elems;
    int* counters;
    int nbins;
};

template <int W>
__global__ void __launch_bounds__(kThreads) spread_kernel(SpreadArgs a) {
    constexpr int W3 = W * W * W;
    constexpr int NIT = (W3 + 31) / 32;
    extern __shared__ float2 tile[];   // [nk][P]
    __shared__ int s_last;
    const Geo& g = a.g;
    const SubProb sp = a.subs[blockIdx.x];
    const int b = blockIdx.y;
    const int P = a.bs1 * a.bs2 * a.bs3;
    const int nk = a.nk;
    const int bin3 = sp.bin % a.nb3;
    const int bt = sp.bin / a.nb3;
    const int bin2 = bt % a.nb2;
    const int bin1 = bt / a.nb2;
    const int lo1 = bin1 * a.bs1, lo2 = bin2 * a.bs2, lo3 = bin3 * a.bs3;
    const int M1 = g.M[0], M2 = g.M[1], M3 = g.M[2];
    const long long G = (long long)M1 * M2 * M3;

    for (int e = threadIdx.x; e < nk * P; e += blockDim.x) tile[e] = make_float2(0.f, 0.f);
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarp = blockDim.x >> 5;
    const float2* yb = a.y + (long long)b * g.J;
    for (int i = warp; i < sp.count; i += nwarp) {
        const int s = __ldg(a.inc + sp.start + i);
        const float4 p = __ldg(a.pts + s);
        const int orig = __float_as_int(p.w);
        const int t = __ldg(a.tframe + s);
        float2 r = __ldg(yb + orig);
        if (a.scale) {
            const float sc = __ldg(a.scale);
            r.x *= sc;
            r.y *= sc;
        }
        const int m01 = (int)ceilf(p.x - g.halfW);
        const int m02 = (int)ceilf(p.y - g.halfW);
        const int m03 = (int)ceilf(p.z - g.halfW);
        float wv = 0.f;
        if (lane < 3 * W) {
            const int d = lane / W, aa = lane - d * W;
            const float gd = d == 0 ? p.x : (d == 1 ? p.y : p.z);
            const int m0 = d == 0 ? m01 : (d == 1 ? m02 : m03);
            const float u = gd - (float)(m0 + aa);
            const float q = 2.f * u / (float)W;
            const float tt = fmaxf(1.f - q * q, 0.f);
            wv = cyl_bessel_i0f(g.beta * sqrtf(tt)) * g.inv_i0_beta;
        }
        // c_k = conj(V[t, k]) r for the channels of this call
        float2 cv[kMaxK];
        const float2* Vt = a.V + (long long)t * g.K + a.k0;
#pragma unroll
        for (int kk = 0; kk < kMaxK; ++kk) {
            if (kk < nk) {
                const float2 v = __ldg(Vt + kk);
                cv[kk] = make_float2(v.x * r.x + v.y * r.y, v.x * r.y - v.y * r.x);
            }
        }
#pragma unroll
        for (int it = 0; it < NIT; ++it) {
            const int tau = lane + 32 * it;
            const bool valid = tau < W3;
            const int tc = valid ? tau : 0;
            const int a1 = tc / (W * W), a2 = (tc / W) % W, a3 = tc % W;
            const float w1 = __shfl_sync(kFull, wv, a1);
            const float w2 = __shfl_sync(kFull, wv, W + a2);
            const float w3 = __shfl_sync(kFull, wv, 2 * W + a3);
            const int i1 = wrap1(m01 + a1, M1) - lo1;
            const int i2 = wrap1(m02 + a2, M2) - lo2;
            const int i3 = wrap1(m03 + a3, M3) - lo3;
            const bool inside = valid && (unsigned)i1 < (unsigned)a.bs1 && (unsigned)i2 < (unsigned)a.bs2 &&
                                (unsigned)i3 < (unsigned)a.bs3;
            if (inside) {
                const float w = w1 * w2 * w3;
                const int l = (i1 * a.bs2 + i2) * a.bs3 + i3;
#pragma unroll
                for (int kk = 0; kk < kMaxK; ++kk) {
                    if (kk < nk) {
                        atomicAdd(&tile[kk * P + l].x, w * cv[kk].x);
                        atomicAdd(&tile[kk * P + l].y, w * cv[kk].y);
                    }
                }
            }
        }
    }
    __syncthreads();

    float2* gb = a.grids + (long long)b * nk * G;
    if (sp.nchunks == 1) {
        for (int e = threadIdx.x; e < nk * P; e += blockDim.x) {
            const int kk = e / P, l = e - kk * P;
            const int x3 = l % a.bs3, x12 = l / a.bs3;
            const int x2 = x12 % a.bs2, x1 = x12 / a.bs2;
            const int j1 = lo1 + x1, j2 = lo2 + x2, j3 = lo3 + x3;
            if (j1 < M1 && j2 < M2 && j3 < M3) gb[kk * G + ((long long)j1 * M2 + j2) * M3 + j3] = tile[e];
        }
        return;
    }
    float2* part = a.partials + ((long long)b * a.slots_per_b + sp.slot + sp.chunk) * a.slot_elems;
    for (int e = threadIdx.x; e < nk * P; e += blockDim.x) part[e] = tile[e];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const int prev = atomicAdd(a.counters + (long long)b * a.nbins + sp.bin, 1);
        s_last = (prev == sp.nchunks - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    const float2* part0 = a.partials + ((long long)b * a.slots_per_b + sp.slot) * a.slot_elems;
    for (int e = threadIdx.x; e < nk * P; e += blockDim.x) {
        float sx = 0.f, sy = 0.f;
        for (int ch = 0; ch < sp.nchunks; ++ch) {
            const float2 v = __ldcg(part0 + (long long)ch * a.slot_elems + e);
            sx += v.x;
            sy += v.y;
        }
        const int kk = e / P, l = e - kk * P;
        const int x3 = l % a.bs3, x12 = l / a.bs3;
        const int x2 = x12 % a.bs2, x1 = x12 / a.bs2;
        const int j1 = lo1 + x1, j2 = lo2 + x2, j3 = lo3 + x3;
        if (j1 < M1 && j2 < M2 && j3 < M3)
            gb[kk * G + ((long long)j1 * M2 + j2) * M3 + j3] = make_float2(sx, sy);
    }
    if (threadIdx.x == 0) a.counters[(long long)b * a.nbins + sp.bin] = 0;
}

template <int W>
cudaError_t launch_w(const SpreadArgs& a, int nsub, int B, size_t smem, cudaStream_t st) {
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(spread_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((unsigned)nsub, (unsigned)B);
    spread_kernel<W><<<grid, kThreads, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_spread(const Geo& g, const int bs[3], const int nb[3], const SubProb* subs, int nsub,
                          const int* inc, const float4* pts, const int* tframe, const float2* V,
                          const float2* y, const float* scale, int B, int k0, int nk, float2* grids,
                          float2* partials, long long slots_per_b, int* counters, int nbins, cudaStream_t st) {
    SpreadArgs a;
    a.g = g;
    a.bs1 = bs[0];
    a.bs2 = bs[1];
    a.bs3 = bs[2];
    a.nb1 = nb[0];
    a.nb2 = nb[1];
    a.nb3 = nb[2];
    a.subs = subs;
    a.inc = inc;
    a.pts = pts;
    a.tframe = tframe;
    a.V = V;
    a.y = y;
    a.scale = scale;
    a.k0 = k0;
    a.nk = nk;
    a.grids = grids;
    a.partials = partials;
    a.slots_per_b = slots_per_b;
    a.slot_elems = (long long)g.K * bs[0] * bs[1] * bs[2];
    a.counters = counters;
    a.nbins = nbins;
    const size_t smem = (size_t)nk * bs[0] * bs[1] * bs[2] * sizeof(float2);
    switch (g.W) {
        case 2: return launch_w<2>(a, nsub, B, smem, st);
        case 3: return launch_w<3>(a, nsub, B, smem, st);
        case 4: return launch_w<4>(a, nsub, B, smem, st);
        case 5: return launch_w<5>(a, nsub, B, smem, st);
        case 6: return launch_w<6>(a, nsub, B, smem, st);
        case 7: return launch_w<7>(a, nsub, B, smem, st);
        case 8: return launch_w<8>(a, nsub, B, smem, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sdp
