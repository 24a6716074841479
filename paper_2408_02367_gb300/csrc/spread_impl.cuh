// Adjoint spreading (kernel template, included by spread.cu and spread_b4.cu) with the conjugate subspace weights (gridding step A5):
//
//   H_{b,k}[m mod M] = sum_j phi(g_j1 - m1) phi(g_j2 - m2) phi(g_j3 - m3) conj(V[t_j, k]) r_b[j]
//
// the first step of A_c^H, which Algorithm 1 of StoDIP needs for
// loss.backward() (Sec. 2.1, Eq. 3).  conj(V[t_j, k]) r_b[j] folds the
// temporal subspace into the spread, so only K channel grids are formed.
//
// Owner-computes bins.  The grid is cut into bins of 8 x 4 x 8 points.  The
// plan lists, per bin, every sample whose W^3 window touches the bin (the
// incidences), split into chunks of bounded length (the subproblems).  A CTA
// is ONE warp that takes one subproblem for one coil b; lane l owns the
// axis-3 column (l / 4, l % 4) of the bin and accumulates its 8 points x the
// channels of the call in registers:
//   - incidences are staged 32 at a time (window start, the 3W plan-time
//     Kaiser-Bessel weights, c_k = conj(V[t, k]) r) in shared memory;
//   - for each incidence a lane multiplies its two axis-1/axis-2 weights and
//     adds w phi3 c_k into the axis-3 positions the window covers;
//   - single-chunk bin: the columns are stored straight into the grid;
//     multi-chunk bin (the dense k-space centre): each chunk stores a partial
//     tile and the last chunk to finish (device-scope counter, no waiting)
//     sums the partials in chunk order and stores the bin.
// Every grid point is written exactly once by plain stores: no zero fill of
// the grid, no atomics on it and no shared-memory accumulation.  The grid is
// channel-interleaved ([b][i1][i2][i3][kk]), so a lane's column of B3 points x
// nk channels is one contiguous run, stored 16 bytes at a time when the call's
// channels form one group.
#pragma once

#include "sdp_internal.cuh"

namespace sdp {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// Bins are 8 x 4 x B3 grid points (axis 1 x axis 2 x axis 3; B3 = 8 or 4).
// Lane l of the warp owns the axis-3 column (x1, x2) = (l / 4, l % 4) of the
// bin: its B3 points x NK channels are accumulated in REGISTERS, so there is no shared
// tile, no load-add-store chain and no bank conflict.  Per incidence a lane
// forms w12 = phi1(x1) phi2(x2) (zero outside the window) and then, for the
// axis-3 positions the window covers (a warp-uniform test), adds
// w12 phi3(x3) conj(V[t, k]) r into acc[x3][k].
constexpr int B1 = 8, B2 = 4;   // the 32 lane columns of a bin; B3 (column depth) is a template parameter

// Two packed (Re, Im) accumulators as one float4 (Re0, Im0, Re1, Im1).
__device__ __forceinline__ float4 pair4(unsigned long long a, unsigned long long b) {
    float4 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(a));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.z), "=f"(r.w) : "l"(b));
    return r;
}

__device__ __forceinline__ unsigned long long pack2(float x, float y) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
    return r;
}

// Store the bin: lane l's column (x1, x2) = (l / 4, l % 4) holds v[x3][q], which
// goes to gbin[x1 cs1 + x2 cs2 + x3 nk + q] for x1 < n1, x2 < n2, x3 < x3end.
// With all nk channels in this group the column's B3 NK values are contiguous:
// the lanes first write their columns to shared memory (tr, CQ 16-byte pairs
// each at an odd stride TS, so a quarter-warp's 16-byte writes hit distinct
// banks), then the warp stores pair e of column e / CQ for e = lane, lane + 32,
// ..., so consecutive lanes write consecutive pieces of one column run (a
// store instruction covers whole runs instead of 32 lines).  All 16-byte
// aligned: M3, lo3 and x3end are even, so a pair never straddles x3end.
// Otherwise (channel groups) each lane stores its own column, 8 bytes at a time.
template <int B3, int NK>
__device__ __forceinline__ void store_bin(float4* tr, const unsigned long long (&v)[B3][NK], float2* gbin,
                                          long long cs1, long long cs2, int n1, int n2, int x3end, int nk,
                                          int lane) {
    constexpr int CQ = B3 * NK / 2;
    constexpr int TS = CQ | 1;
    if (NK == nk) {
        __syncwarp();
#pragma unroll
        for (int j = 0; j < CQ; ++j)
            tr[lane * TS + j] = pair4(v[(2 * j) / NK][(2 * j) % NK], v[(2 * j + 1) / NK][(2 * j + 1) % NK]);
        __syncwarp();
#pragma unroll
        for (int r = 0; r < CQ; ++r) {
            const int e = r * 32 + lane;
            const int c = e / CQ, j = e - c * CQ;
            const int c1 = c >> 2, c2 = c & 3;
            if (c1 < n1 && c2 < n2 && 2 * j < x3end * NK)
                *reinterpret_cast<float4*>(gbin + c1 * cs1 + c2 * cs2 + 2 * j) = tr[c * TS + j];
        }
    } else {
        const int x1 = lane >> 2, x2 = lane & 3;
        if (x1 < n1 && x2 < n2) {
            float2* gcol = gbin + x1 * cs1 + x2 * cs2;
#pragma unroll
            for (int x3 = 0; x3 < B3; ++x3)
                if (x3 < x3end)
#pragma unroll
                    for (int q = 0; q < NK; ++q)
                        *reinterpret_cast<unsigned long long*>(gcol + (long long)x3 * nk + q) = v[x3][q];
        }
    }
}

// One warp's unit: subproblem `sub` for coils NC * by .. NC * by + NC - 1 (those below B).
template <int B3, int W, int NK, int NC>
__device__ __forceinline__ void spread_body(const SpreadArgs& a, int kofs, int B, int sub, int by) {
    constexpr int BP = B1 * B2 * B3;
    constexpr int NW = 3 * W;
    constexpr int NP = B1 + B2;               // staged axis-1 and axis-2 weights per incidence
    // staging of 32 incidences, reused for the bin's store once they are summed.  Every
    // lane reads each incidence's record (a broadcast), and a 16-byte shared load costs
    // two L1 wavefronts, so the records are packed: the B3 axis-3 weights as plain floats
    // (the (w3, w3) pairs are formed in registers), and the coefficients conj(V[t, k]) r_b
    // of all NC coils of the warp (NC = 2: the positions, weights and coverage of an
    // incidence are staged once and serve both coils) in one run of NCK values, padded
    // to an even count so that it is read 16 bytes at a time.
    constexpr int NCK = NC * NK;
    constexpr int NCKP = (NCK + 1) & ~1;
    constexpr int kStage = 32 * B3 * 4 + 32 * NCKP * 8 + 32 * NP * 4 + 32 * 4;
    constexpr int kTr = 32 * ((B3 * NK / 2) | 1) * 16;
    __shared__ __align__(16) unsigned char sraw[kStage > kTr ? kStage : kTr];
    float* p3f = reinterpret_cast<float*>(sraw);       // [incidence][x3]: w3, 0 outside the window
    float2* csm = reinterpret_cast<float2*>(p3f + 32 * B3);   // [incidence][coil][k]: conj(V[t, k]) r_b
    float* psm = reinterpret_cast<float*>(csm + 32 * NCKP);   // [incidence][x1 (8) | x2 (4)], 0 outside
    unsigned* msm = reinterpret_cast<unsigned*>(psm + 32 * NP);   // axis-3 positions covered (bit x3)
    float4* tr = reinterpret_cast<float4*>(sraw);
    const Geo& g = a.g;
    const int lane = threadIdx.x;
    const int x1 = lane >> 2, x2 = lane & 3;
    const SubProb sp = a.subs[sub];
    const int b0 = by * NC;                            // first coil of the warp
    const int nc = min(NC, B - b0);                    // its coils (the last warp of an odd batch has one)
    const int bin3 = sp.bin % a.nb3;
    const int bt = sp.bin / a.nb3;
    const int bin2 = bt % a.nb2;
    const int bin1 = bt / a.nb2;
    const int lo1 = bin1 * B1, lo2 = bin2 * B2, lo3 = bin3 * B3;
    const int M1 = g.M[0], M2 = g.M[1], M3 = g.M[2];
    const long long G = (long long)M1 * M2 * M3;

    // accumulators as packed (Re, Im) pairs for the f32x2 multiply-adds
    unsigned long long acc[NC][B3][NK];
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int x3 = 0; x3 < B3; ++x3)
#pragma unroll
            for (int q = 0; q < NK; ++q) acc[c][x3][q] = 0ull;

    const float sc = a.scale ? __ldg(a.scale) : 1.f;
    const int kv = a.k0 + kofs;   // first channel of V of this group
    for (int base = 0; base < sp.count; base += 32) {
        const int n = min(32, sp.count - base);
        if (lane < n) {
            const int s = __ldg(a.inc + sp.start + base + lane);
            const float4 p = __ldg(a.pts + s);
            const int orig = __float_as_int(p.w);
            const int t = __ldg(a.tframe + s);
            const float* ws = a.wts + (long long)s * NW;
            float wl[NW];
#pragma unroll
            for (int q = 0; q < NW; ++q) wl[q] = __ldg(ws + q);
            // tap offset of every bin position, wrapped onto the periodic grid:
            // position x takes weight phi_d(a) with a = (lo + x - m0) mod M if a < W
            const int m01 = (int)ceilf(p.x - g.halfW), m02 = (int)ceilf(p.y - g.halfW);
            const int m03 = (int)ceilf(p.z - g.halfW);
            float* pw = psm + lane * NP;
#pragma unroll
            for (int x = 0; x < B1; ++x) {
                int aa = lo1 + x - m01;
                aa += aa < 0 ? M1 : 0;
                aa -= aa >= M1 ? M1 : 0;
                float v = 0.f;
#pragma unroll
                for (int q = 0; q < W; ++q) v = aa == q ? wl[q] : v;
                pw[x] = v;
            }
#pragma unroll
            for (int x = 0; x < B2; ++x) {
                int aa = lo2 + x - m02;
                aa += aa < 0 ? M2 : 0;
                aa -= aa >= M2 ? M2 : 0;
                float v = 0.f;
#pragma unroll
                for (int q = 0; q < W; ++q) v = aa == q ? wl[W + q] : v;
                pw[B1 + x] = v;
            }
            unsigned mask = 0;
            float w3v[B3];
#pragma unroll
            for (int x = 0; x < B3; ++x) {
                int aa = lo3 + x - m03;
                aa += aa < 0 ? M3 : 0;
                aa -= aa >= M3 ? M3 : 0;
                float v = 0.f;
#pragma unroll
                for (int q = 0; q < W; ++q) v = aa == q ? wl[2 * W + q] : v;
                w3v[x] = v;
                mask |= ((unsigned)aa < (unsigned)W ? 1u : 0u) << x;
            }
#pragma unroll
            for (int x = 0; x < B3; x += 4)
                *reinterpret_cast<float4*>(p3f + lane * B3 + x) = make_float4(w3v[x], w3v[x + 1], w3v[x + 2], w3v[x + 3]);
            msm[lane] = mask;
            const float2* Vt = a.V + (long long)t * g.K + kv;
            float2 vq[NK];
#pragma unroll
            for (int q = 0; q < NK; ++q) vq[q] = __ldg(Vt + q);
            float2 cv[NCKP];
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                float2 r = make_float2(0.f, 0.f);   // a missing second coil spreads zeros and is not stored
                if (c < nc) {
                    r = __ldg(a.y + (long long)(b0 + c) * g.J + orig);
                    r.x *= sc;
                    r.y *= sc;
                }
#pragma unroll
                for (int q = 0; q < NK; ++q)
                    cv[c * NK + q] = make_float2(vq[q].x * r.x + vq[q].y * r.y, vq[q].x * r.y - vq[q].y * r.x);
            }
            if (NCKP > NCK) cv[NCKP - 1] = make_float2(0.f, 0.f);
#pragma unroll
            for (int q = 0; q < NCKP; q += 2)
                *reinterpret_cast<float4*>(csm + lane * NCKP + q) = make_float4(cv[q].x, cv[q].y, cv[q + 1].x, cv[q + 1].y);
        }
        __syncwarp();
        for (int i = 0; i < n; ++i) {
            const float* pw = psm + i * NP;
            const unsigned mask = msm[i];
            const float w12 = pw[x1] * pw[B1 + x2];
            unsigned long long w12p;
            asm("mov.b64 %0, {%1, %1};" : "=l"(w12p) : "f"(w12));
            const float4* wp = reinterpret_cast<const float4*>(p3f + i * B3);
            const ulonglong2* cp = reinterpret_cast<const ulonglong2*>(csm + i * NCKP);
            unsigned long long cf[NCKP], wp3[B3];
#pragma unroll
            for (int q = 0; q < NCKP / 2; ++q) {
                const ulonglong2 v = cp[q];
                cf[2 * q] = v.x;
                cf[2 * q + 1] = v.y;
            }
#pragma unroll
            for (int x3 = 0; x3 < B3 / 4; ++x3) {
                const float4 v = wp[x3];
                asm("mov.b64 %0, {%1, %1};" : "=l"(wp3[4 * x3]) : "f"(v.x));
                asm("mov.b64 %0, {%1, %1};" : "=l"(wp3[4 * x3 + 1]) : "f"(v.y));
                asm("mov.b64 %0, {%1, %1};" : "=l"(wp3[4 * x3 + 2]) : "f"(v.z));
                asm("mov.b64 %0, {%1, %1};" : "=l"(wp3[4 * x3 + 3]) : "f"(v.w));
            }
#pragma unroll
            for (int x3 = 0; x3 < B3; ++x3) {
                if (mask & (1u << x3)) {                 // the same for every lane
                    // w = w12 * w3 and acc += w * c, both components at once (round to nearest
                    // per component: the same arithmetic as two scalar multiplies and FMAs)
                    unsigned long long w;
                    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(w) : "l"(w12p), "l"(wp3[x3]));
#pragma unroll
                    for (int c = 0; c < NC; ++c)
#pragma unroll
                        for (int q = 0; q < NK; ++q)
                            asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc[c][x3][q]) : "l"(w), "l"(cf[c * NK + q]));
                }
            }
        }
        __syncwarp();
    }

    // store: column (x1, x2) of the bin, element (x3, q) at gbin[x1 cs1 + x2 cs2 + x3 nk + q]
    const int nk = a.nk;
    const long long cs2 = (long long)M3 * nk, cs1 = (long long)M2 * cs2;
    float2* gbin0 = a.grids + (long long)b0 * G * nk + (((long long)lo1 * M2 + lo2) * M3 + lo3) * nk + kofs;
    const int n1 = M1 - lo1, n2 = M2 - lo2;
    const int x3end = min(B3, M3 - lo3);
    if (sp.nchunks == 1) {
#pragma unroll
        for (int c = 0; c < NC; ++c)
            if (c < nc)
                store_bin<B3, NK>(tr, acc[c], gbin0 + (long long)c * G * nk, cs1, cs2, n1, n2, x3end, nk, lane);
        return;
    }
    // multi-chunk bin: the chunk's partial tile of each coil in its slot, 16-byte pair j of
    // lane l at [j][l] (each store instruction writes 512 contiguous bytes); the last chunk
    // to arrive (one counter per bin and first coil of the warp) sums them
    constexpr int CQ = B3 * NK / 2;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        if (c < nc) {
            float4* part = reinterpret_cast<float4*>(
                a.partials + ((long long)(b0 + c) * a.slots_per_b + sp.slot + sp.chunk) * a.slot_elems +
                (long long)kofs * BP);
#pragma unroll
            for (int j = 0; j < CQ; ++j)
                part[j * 32 + lane] =
                    pair4(acc[c][(2 * j) / NK][(2 * j) % NK], acc[c][(2 * j + 1) / NK][(2 * j + 1) % NK]);
        }
    }
    __threadfence();
    __syncwarp();
    int last = 0;
    int* counter = a.counters + ((long long)b0 * a.ngroups + a.group) * a.nbins + sp.bin;
    if (lane == 0) last = (atomicAdd(counter, 1) == sp.nchunks - 1);
    last = __shfl_sync(kFull, last, 0);
    if (!last) return;
    __threadfence();
    const long long slot4 = a.slot_elems / 2;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        if (c < nc) {
            const float4* part0 = reinterpret_cast<const float4*>(
                a.partials + ((long long)(b0 + c) * a.slots_per_b + sp.slot) * a.slot_elems + (long long)kofs * BP);
#pragma unroll
            for (int j = 0; j < CQ; ++j) {
                float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
                for (int ch = 0; ch < sp.nchunks; ++ch) {
                    const float4 v = __ldcg(part0 + ch * slot4 + j * 32 + lane);
                    sum.x += v.x;
                    sum.y += v.y;
                    sum.z += v.z;
                    sum.w += v.w;
                }
                acc[c][(2 * j) / NK][(2 * j) % NK] = pack2(sum.x, sum.y);
                acc[c][(2 * j + 1) / NK][(2 * j + 1) % NK] = pack2(sum.z, sum.w);
            }
            store_bin<B3, NK>(tr, acc[c], gbin0 + (long long)c * G * nk, cs1, cs2, n1, n2, x3end, nk, lane);
        }
    }
    if (lane == 0) *counter = 0;
}

template <int B3, int W, int NK, int NC>
__global__ void __launch_bounds__(32, NC * B3 * NK <= 20 ? 24 : (NC * B3 * NK <= 40 ? 16 : 1))
spread_kernel(SpreadArgs a, int kofs, int B) {
    spread_body<B3, W, NK, NC>(a, kofs, B, (int)blockIdx.x, (int)blockIdx.y);
}

// Coils per warp: two where the doubled accumulators fit (4-deep columns of at most 5
// channels: 40 packed pairs), else one.
template <int B3, int NK>
__host__ __device__ constexpr int spread_coils() { return spread_pairs_fit(B3, NK) ? 2 : 1; }

template <int B3, int W, int NK>
cudaError_t launch_wk(const SpreadArgs& a, int kofs, int nsub, int B, int coils, cudaStream_t st) {
    constexpr int NC2 = spread_coils<B3, NK>();
    if (NC2 == 2 && coils != 1 && B >= 2) {
        dim3 grid((unsigned)nsub, (unsigned)((B + 1) / 2));
        spread_kernel<B3, W, NK, NC2><<<grid, 32, 0, st>>>(a, kofs, B);
    } else {
        dim3 grid((unsigned)nsub, (unsigned)B);
        spread_kernel<B3, W, NK, 1><<<grid, 32, 0, st>>>(a, kofs, B);
    }
    return cudaGetLastError();
}

// Channels run in groups of at most 8 (one launch each, exact group size).
template <int B3, int W>
cudaError_t launch_w(SpreadArgs a, int nsub, int B, int coils, cudaStream_t st) {
    if (a.bs1 != B1 || a.bs2 != B2 || a.bs3 != B3) return cudaErrorInvalidValue;
    a.ngroups = (a.nk + 7) / 8;
    for (int gi = 0; gi < a.ngroups; ++gi) {
        const int kofs = gi * 8;
        const int ng = a.nk - kofs < 8 ? a.nk - kofs : 8;
        a.group = gi;
        cudaError_t e;
        switch (ng) {
            case 1: e = launch_wk<B3, W, 1>(a, kofs, nsub, B, coils, st); break;
            case 2: e = launch_wk<B3, W, 2>(a, kofs, nsub, B, coils, st); break;
            case 3: e = launch_wk<B3, W, 3>(a, kofs, nsub, B, coils, st); break;
            case 4: e = launch_wk<B3, W, 4>(a, kofs, nsub, B, coils, st); break;
            case 5: e = launch_wk<B3, W, 5>(a, kofs, nsub, B, coils, st); break;
            case 6: e = launch_wk<B3, W, 6>(a, kofs, nsub, B, coils, st); break;
            case 7: e = launch_wk<B3, W, 7>(a, kofs, nsub, B, coils, st); break;
            default: e = launch_wk<B3, W, 8>(a, kofs, nsub, B, coils, st); break;
        }
        if (e != cudaSuccess) return e;
        if (gi > 0) note_launches(1);   // the stage counts its first launch
    }
    return cudaSuccess;
}

template <int B3>
cudaError_t launch_spread_depth(const Geo& g, const int bs[3], const int nb[3], const SubProb* subs, int nsub,
                          const int* inc, const float4* pts, const int* tframe, const float* wts, const float2* V,
                          const float2* y, const float* scale, int B, int k0, int nk, float2* grids,
                          float2* partials, long long slots_per_b, int* counters, int nbins, int coils,
                          cudaStream_t st) {
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
    a.ngroups = 1;
    a.group = 0;
    switch (g.W) {
        case 2: return launch_w<B3, 2>(a, nsub, B, coils, st);
        case 3: return launch_w<B3, 3>(a, nsub, B, coils, st);
        case 4: return launch_w<B3, 4>(a, nsub, B, coils, st);
        case 5: return launch_w<B3, 5>(a, nsub, B, coils, st);
        case 6: return launch_w<B3, 6>(a, nsub, B, coils, st);
        case 7: return launch_w<B3, 7>(a, nsub, B, coils, st);
        case 8: return launch_w<B3, 8>(a, nsub, B, coils, st);
        default: return cudaErrorInvalidValue;
    }
}


}  // namespace
}  // namespace sdp
