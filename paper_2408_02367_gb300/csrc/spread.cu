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
// is ONE warp that takes one subproblem for one coil b and owns a private
// shared-memory tile of the bin (all K channels):
//   - incidences are staged 32 at a time (sample index, window start, the 3W
//     plan-time Kaiser-Bessel weights, c_k = conj(V[t, k]) r) in shared memory;
//   - each incidence is then spread with lanes over its W^3 taps.  Within one
//     warp instruction the lanes touch distinct tile points and no other warp
//     touches the tile, so the accumulation is a plain shared load-add-store:
//     no atomics at all;
//   - single-chunk bin: the tile is stored straight into the grid;
//     multi-chunk bin (the dense k-space centre): each chunk stores a partial
//     tile and the last chunk to finish (device-scope counter, no waiting)
//     sums the partials in chunk order and stores the bin.
// Every grid point is written exactly once by plain 16-byte stores: no zero
// fill of the grid and no global atomics on it.
#include "sdp_internal.cuh"

namespace sdp {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int wrap1(int i, int M) { return i < 0 ? i + M : (i >= M ? i - M : i); }

struct SpreadArgs {
    Geo g;
    int bs1, bs2, bs3;
    int nb1, nb2, nb3;
    const SubProb* subs;
    const int* inc;
    const float4* pts;
    const int* tframe;
    const float* wts;
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

// Channel groups: CK channels are handled per pass over an incidence's taps
// (CK is a compile-time constant so the channel loop fully unrolls without
// predicated dead slots); nk > CK runs ceil(nk / CK) groups, the last one masked.
template <int W, int CK>
__global__ void __launch_bounds__(32) spread_kernel(SpreadArgs a) {
    constexpr int W3 = W * W * W;
    constexpr int NIT = (W3 + 31) / 32;
    constexpr int NW = 3 * W;
    extern __shared__ float4 smem4[];
    const Geo& g = a.g;
    const int nk = a.nk;
    const int P = a.bs1 * a.bs2 * a.bs3;
    float2* tile = reinterpret_cast<float2*>(smem4);            // [nk][P]
    float* wsm = reinterpret_cast<float*>(tile + nk * P);       // [32][NW]
    float2* csm = reinterpret_cast<float2*>(wsm + 32 * NW);     // [32][nk]
    int* dsm = reinterpret_cast<int*>(csm + 32 * nk);           // [32][4]

    const int lane = threadIdx.x;
    const SubProb sp = a.subs[blockIdx.x];
    const int b = blockIdx.y;
    const int bin3 = sp.bin % a.nb3;
    const int bt = sp.bin / a.nb3;
    const int bin2 = bt % a.nb2;
    const int bin1 = bt / a.nb2;
    const int lo1 = bin1 * a.bs1, lo2 = bin2 * a.bs2, lo3 = bin3 * a.bs3;
    const int M1 = g.M[0], M2 = g.M[1], M3 = g.M[2];
    const long long G = (long long)M1 * M2 * M3;
    const int s23 = a.bs2 * a.bs3;

    // taps owned by this lane and their offset inside the tile relative to the window start
    int ta1[NIT], ta2[NIT], ta3[NIT], toff[NIT];
    bool tv[NIT];
#pragma unroll
    for (int it = 0; it < NIT; ++it) {
        const int tau = lane + 32 * it;
        tv[it] = tau < W3;
        const int tc = tv[it] ? tau : 0;
        ta1[it] = tc / (W * W);
        ta2[it] = (tc / W) % W;
        ta3[it] = tc % W;
        toff[it] = ta1[it] * s23 + ta2[it] * a.bs3 + ta3[it];
    }

    float4* tile4 = reinterpret_cast<float4*>(tile);
    const int n4 = nk * P / 2;
    for (int e = lane; e < n4; e += 32) tile4[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncwarp();

    const float2* yb = a.y + (long long)b * g.J;
    const float sc = a.scale ? __ldg(a.scale) : 1.f;
    for (int base = 0; base < sp.count; base += 32) {
        const int n = min(32, sp.count - base);
        if (lane < n) {
            const int s = __ldg(a.inc + sp.start + base + lane);
            const float4 p = __ldg(a.pts + s);
            const int orig = __float_as_int(p.w);
            const int t = __ldg(a.tframe + s);
            float2 r = __ldg(yb + orig);
            r.x *= sc;
            r.y *= sc;
            const int m01 = (int)ceilf(p.x - g.halfW);
            const int m02 = (int)ceilf(p.y - g.halfW);
            const int m03 = (int)ceilf(p.z - g.halfW);
            const bool nowrap = m01 >= 0 && m01 + W <= M1 && m02 >= 0 && m02 + W <= M2 && m03 >= 0 && m03 + W <= M3;
            dsm[lane * 4 + 0] = m01 - lo1;
            dsm[lane * 4 + 1] = m02 - lo2;
            dsm[lane * 4 + 2] = m03 - lo3;
            dsm[lane * 4 + 3] = nowrap ? 1 : 0;
            const float* ws = a.wts + (long long)s * NW;
#pragma unroll
            for (int q = 0; q < NW; ++q) wsm[lane * NW + q] = __ldg(ws + q);
            const float2* Vt = a.V + (long long)t * g.K + a.k0;
            for (int kk = 0; kk < nk; ++kk) {
                const float2 v = __ldg(Vt + kk);
                csm[lane * nk + kk] = make_float2(v.x * r.x + v.y * r.y, v.x * r.y - v.y * r.x);
            }
        }
        __syncwarp();
        for (int i = 0; i < n; ++i) {
            const int4 dd = *reinterpret_cast<const int4*>(dsm + i * 4);
            const float wv = lane < NW ? wsm[i * NW + lane] : 0.f;
            const int dbase = dd.x * s23 + dd.y * a.bs3 + dd.z;
            float w[NIT];
            int l[NIT];
            bool in[NIT];
#pragma unroll
            for (int it = 0; it < NIT; ++it) {
                const float w1 = __shfl_sync(kFull, wv, ta1[it]);
                const float w2 = __shfl_sync(kFull, wv, W + ta2[it]);
                const float w3 = __shfl_sync(kFull, wv, 2 * W + ta3[it]);
                w[it] = w1 * w2 * w3;
                int x1 = dd.x + ta1[it], x2 = dd.y + ta2[it], x3 = dd.z + ta3[it];
                l[it] = dbase + toff[it];
                if (!dd.w) {   // the window wraps around the grid edge (rare): wrap every tap
                    x1 = wrap1(dd.x + lo1 + ta1[it], M1) - lo1;
                    x2 = wrap1(dd.y + lo2 + ta2[it], M2) - lo2;
                    x3 = wrap1(dd.z + lo3 + ta3[it], M3) - lo3;
                    l[it] = x1 * s23 + x2 * a.bs3 + x3;
                }
                in[it] = tv[it] && (unsigned)x1 < (unsigned)a.bs1 && (unsigned)x2 < (unsigned)a.bs2 &&
                         (unsigned)x3 < (unsigned)a.bs3;
            }
            for (int k0 = 0; k0 < nk; k0 += CK) {
                float2 c[CK];
#pragma unroll
                for (int q = 0; q < CK; ++q)
                    if (CK == 1 || k0 + q < nk) c[q] = csm[i * nk + k0 + q];
#pragma unroll
                for (int it = 0; it < NIT; ++it) {
                    if (in[it]) {
                        float2* pt = tile + l[it] + k0 * P;
                        float2 o[CK];
#pragma unroll
                        for (int q = 0; q < CK; ++q)
                            if (CK == 1 || k0 + q < nk) o[q] = pt[q * P];
#pragma unroll
                        for (int q = 0; q < CK; ++q) {
                            if (CK == 1 || k0 + q < nk) {
                                o[q].x = fmaf(w[it], c[q].x, o[q].x);
                                o[q].y = fmaf(w[it], c[q].y, o[q].y);
                                pt[q * P] = o[q];
                            }
                        }
                    }
                }
            }
        }
        __syncwarp();
    }

    // store: pairs of points along axis 3 (bs3, M3 and lo3 are even) as one 16-byte store
    float2* gb = a.grids + (long long)b * nk * G;
    const int half3 = a.bs3 / 2;
    if (sp.nchunks == 1) {
        for (int e = lane; e < n4; e += 32) {
            const int kk = e / (P / 2), l2 = e - kk * (P / 2);
            const int x3 = 2 * (l2 % half3), x12 = l2 / half3;
            const int x2 = x12 % a.bs2, x1 = x12 / a.bs2;
            const int j1 = lo1 + x1, j2 = lo2 + x2, j3 = lo3 + x3;
            if (j1 < M1 && j2 < M2 && j3 < M3)
                *reinterpret_cast<float4*>(gb + kk * G + ((long long)j1 * M2 + j2) * M3 + j3) = tile4[e];
        }
        return;
    }
    float4* part = reinterpret_cast<float4*>(a.partials +
                                             ((long long)b * a.slots_per_b + sp.slot + sp.chunk) * a.slot_elems);
    for (int e = lane; e < n4; e += 32) part[e] = tile4[e];
    __threadfence();
    __syncwarp();
    int last = 0;
    if (lane == 0) last = (atomicAdd(a.counters + (long long)b * a.nbins + sp.bin, 1) == sp.nchunks - 1);
    last = __shfl_sync(kFull, last, 0);
    if (!last) return;
    __threadfence();
    const float4* part0 =
        reinterpret_cast<const float4*>(a.partials + ((long long)b * a.slots_per_b + sp.slot) * a.slot_elems);
    const long long slot4 = a.slot_elems / 2;
    for (int e = lane; e < n4; e += 32) {
        float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int ch = 0; ch < sp.nchunks; ++ch) {
            const float4 v = __ldcg(part0 + ch * slot4 + e);
            s.x += v.x;
            s.y += v.y;
            s.z += v.z;
            s.w += v.w;
        }
        const int kk = e / (P / 2), l2 = e - kk * (P / 2);
        const int x3 = 2 * (l2 % half3), x12 = l2 / half3;
        const int x2 = x12 % a.bs2, x1 = x12 / a.bs2;
        const int j1 = lo1 + x1, j2 = lo2 + x2, j3 = lo3 + x3;
        if (j1 < M1 && j2 < M2 && j3 < M3)
            *reinterpret_cast<float4*>(gb + kk * G + ((long long)j1 * M2 + j2) * M3 + j3) = s;
    }
    if (lane == 0) a.counters[(long long)b * a.nbins + sp.bin] = 0;
}

template <int W, int CK>
cudaError_t launch_wk(const SpreadArgs& a, int nsub, int B, cudaStream_t st) {
    const size_t smem = (size_t)a.nk * a.bs1 * a.bs2 * a.bs3 * sizeof(float2) + 32 * 3 * W * sizeof(float) +
                        32 * a.nk * sizeof(float2) + 32 * 4 * sizeof(int);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(spread_kernel<W, CK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((unsigned)nsub, (unsigned)B);
    spread_kernel<W, CK><<<grid, 32, smem, st>>>(a);
    return cudaGetLastError();
}

template <int W>
cudaError_t launch_w(const SpreadArgs& a, int nsub, int B, cudaStream_t st) {
    switch (channel_group(a.nk)) {
        case 1: return launch_wk<W, 1>(a, nsub, B, st);
        case 2: return launch_wk<W, 2>(a, nsub, B, st);
        case 3: return launch_wk<W, 3>(a, nsub, B, st);
        case 4: return launch_wk<W, 4>(a, nsub, B, st);
        case 5: return launch_wk<W, 5>(a, nsub, B, st);
        default: return launch_wk<W, 8>(a, nsub, B, st);
    }
}

}  // namespace

cudaError_t launch_spread(const Geo& g, const int bs[3], const int nb[3], const SubProb* subs, int nsub,
                          const int* inc, const float4* pts, const int* tframe, const float* wts, const float2* V,
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
    a.wts = wts;
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
    switch (g.W) {
        case 2: return launch_w<2>(a, nsub, B, st);
        case 3: return launch_w<3>(a, nsub, B, st);
        case 4: return launch_w<4>(a, nsub, B, st);
        case 5: return launch_w<5>(a, nsub, B, st);
        case 6: return launch_w<6>(a, nsub, B, st);
        case 7: return launch_w<7>(a, nsub, B, st);
        case 8: return launch_w<8>(a, nsub, B, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sdp
