// Adjoint spreading (kernel template, included by the spread_*.cu translation
// units and batch_sp.cu) with the conjugate subspace weights (gridding step A5):
//
//   H_{b,k}[m mod M] = sum_j phi(g_j1 - m1) phi(g_j2 - m2) phi(g_j3 - m3) conj(V[t_j, k]) r_b[j]
//
// the first step of A_c^H, which Algorithm 1 of StoDIP needs for
// loss.backward() (Sec. 2.1, Eq. 3).  conj(V[t_j, k]) r_b[j] folds the
// temporal subspace into the spread, so only K channel grids are formed.
//
// Owner-computes bins.  The grid is cut into bins of B1 x 4 x B3 points
// (B1, B3 = 8 or 4).  The plan lists, per bin, every sample whose W^3 window
// touches the bin (the incidences), ordered by where the window meets the bin
// along axis 3 (the incidence's class, below), and split into chunks of
// bounded length (the subproblems).  A CTA is ONE warp that takes one
// subproblem for NC coils.  The bin's B1 x 4 axis-3 columns belong to lanes,
// and a lane accumulates its column's B3 points x the call's channels x NC
// coils in registers:
//   - B1 = 8: lane l owns column (l / 4, l % 4); the whole warp takes each
//     incidence;
//   - B1 = 4: lanes l and l + 16 own column ((l % 16) / 4, l % 4), and the two
//     half-warps take alternate incidences, adding their registers together at
//     the end.  A window of 4 x 4 columns covers a larger share of a 4 x 4
//     column set than of an 8 x 4 one, so more of every multiply-add counts.
// Incidences are staged 32 at a time in shared memory: per-position axis-1
// and axis-2 weights, the B3 axis-3 weights (zero outside the window) and
// c_k = conj(V[t, k]) r_b for the warp's coils.  For W = 4 and 6 a run of
// incidences of one class runs code compiled for exactly that class's
// positions.  The class is o + W - 1, where o is the bin position of the
// window's first axis-3 tap; the window then covers positions
// [max(0, o), min(B3, o + W)).  There is no per-position test and no
// multiply-add on a position the window misses.  Other widths use every
// position, with zero weights where the window does not reach.  So do grids
// too short along axis 3 for a window to meet a bin in one piece.
// Finishing a bin:
//   - single-chunk bin: the columns are stored straight into the grid;
//   - multi-chunk bin (the dense k-space centre): each chunk stores a partial
//     tile, and the last chunk to finish (device-scope counter, no waiting)
//     sums the partials in chunk order and stores the bin.
// Every grid point is written exactly once by plain stores: no zero fill of
// the grid, no atomics on it and no shared-memory accumulation.  The grid is
// channel-interleaved ([b][i1][i2][i3][kk]), so a column's B3 points x nk
// channels are one contiguous run.  The warp stores the bin through shared
// memory, so consecutive lanes write consecutive 16-byte pieces of those runs.
#pragma once

#include "index_map.cuh"
#include "sdp_internal.cuh"

namespace sdp {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kB2 = 4;     // bin extent along axis 2
constexpr int kNPS = 12;   // staged axis-1 + axis-2 weights per incidence (B1 + 4, padded to 12 floats)

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

__device__ __forceinline__ float2 unpack2(unsigned long long v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}

// Axis-3 classes of a bin of depth B3 for width W: class c = o + W - 1 covers the
// positions [max(0, o), min(B3, o + W)); class kAll covers every position.
template <int B3, int W>
struct Axis3Classes {
    static constexpr bool kOn = (W == 4 || W == 6);
    static constexpr int kAll = kOn ? B3 + W - 1 : 0;
    template <int C>
    __host__ __device__ static constexpr int lo() { return C == kAll ? 0 : (C - (W - 1) > 0 ? C - (W - 1) : 0); }
    template <int C>
    __host__ __device__ static constexpr int hi() { return C == kAll ? B3 : (C + 1 < B3 ? C + 1 : B3); }
};

// Incidences [i, e) of one class, positions [XL, XH) of the lane's column.  With two
// incidences per step (B1 = 4) half-warp h takes incidence j + h; a missing second
// incidence at the end of an odd run adds zero weight to a staged one.
template <int XL, int XH, int B1, int B3, int NK, int NC>
__device__ __forceinline__ void spread_run(unsigned long long (&acc)[NC][B3][NK], const float* psm, const float* p3f,
                                           const float2* csm, int i, int e, int h, int x1, int x2) {
    constexpr int IPW = 32 / (B1 * kB2);
    constexpr int NCKP = (NC * NK + 1) & ~1;
#pragma unroll 1
    for (int j = i; j < e; j += IPW) {
        int ii = j + h;
        bool ok = true;
        if (IPW > 1) {
            ok = ii < e;
            ii = ok ? ii : j;
        }
        const float* pw = psm + ii * kNPS;
        float w12 = pw[x1] * pw[B1 + x2];
        if (IPW > 1) w12 = ok ? w12 : 0.f;
        float w3[B3];
        const float4* wp = reinterpret_cast<const float4*>(p3f + ii * B3);
#pragma unroll
        for (int q = XL / 4; q <= (XH - 1) / 4; ++q) {
            const float4 v = wp[q];
            w3[4 * q] = v.x;
            w3[4 * q + 1] = v.y;
            w3[4 * q + 2] = v.z;
            w3[4 * q + 3] = v.w;
        }
        const ulonglong2* cp = reinterpret_cast<const ulonglong2*>(csm + ii * NCKP);
        unsigned long long cf[NCKP];
#pragma unroll
        for (int q = 0; q < NCKP / 2; ++q) {
            const ulonglong2 v = cp[q];
            cf[2 * q] = v.x;
            cf[2 * q + 1] = v.y;
        }
#pragma unroll
        for (int x3 = XL; x3 < XH; ++x3) {
            // acc += (w12 w3) c, both components at once (round to nearest per component:
            // the same arithmetic as two scalar multiply-adds)
            const float w = w12 * w3[x3];
            unsigned long long wd;
            asm("mov.b64 %0, {%1, %1};" : "=l"(wd) : "f"(w));
#pragma unroll
            for (int c = 0; c < NC; ++c)
#pragma unroll
                for (int q = 0; q < NK; ++q)
                    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc[c][x3][q]) : "l"(wd), "l"(cf[c * NK + q]));
        }
    }
}

// The run of class c: classes C .. N-1 by a chain of tests, any other value as class N
// (every position).  Compile-time recursion, so the accumulators stay in registers.
template <int C, int B1, int B3, int W, int NK, int NC>
__device__ __forceinline__ void spread_class(int c, unsigned long long (&acc)[NC][B3][NK], const float* psm,
                                             const float* p3f, const float2* csm, int i, int e, int h, int x1,
                                             int x2) {
    using Cls = Axis3Classes<B3, W>;
    if constexpr (C < Cls::kAll) {
        if (c == C)
            spread_run<Cls::template lo<C>(), Cls::template hi<C>(), B1, B3, NK, NC>(acc, psm, p3f, csm, i, e, h, x1,
                                                                                      x2);
        else
            spread_class<C + 1, B1, B3, W, NK, NC>(c, acc, psm, p3f, csm, i, e, h, x1, x2);
    } else {
        spread_run<0, B3, B1, B3, NK, NC>(acc, psm, p3f, csm, i, e, h, x1, x2);
    }
}

// Store ncols columns of a bin from shared memory: column cl = s * (B1 4) + c holds
// coil slot s's column c = (c1, c2) = (c / 4, c % 4) as CQ 16-byte pairs at
// tr[cl TS ..], element (x3, q) going to g0[s cstr + c1 cs1 + c2 cs2 + x3 nk + q] for
// c1 < n1, c2 < n2, x3 < x3end.  With all nk channels in this group a column is one
// contiguous run and the warp writes consecutive 16-byte pieces of the runs (16-byte
// aligned: M3, lo3 and x3end are even, so a pair never straddles x3end); otherwise
// (channel groups) 8 bytes at a time.  TS = CQ | 1 is odd, so the quarter-warps that
// move their columns' registers into tr write distinct banks; the reads here meet at
// most two 16-byte slots per bank (where a column's pad slot is skipped).  The index
// maps are in index_map.cuh.
template <int B1, int B3, int NK>
__device__ __forceinline__ void store_cols(const float4* tr, int ncols, float2* g0, long long cstr, long long cs1,
                                           long long cs2, int n1, int n2, int x3end, int nk, int lane) {
    constexpr int NCOL = B1 * kB2;
    constexpr int CQ = imap::spread_cq(B3, NK);
    constexpr int TS = imap::spread_ts(B3, NK);
    if (NK == nk) {
        const int tot = ncols * CQ;
        for (int e = lane; e < tot; e += 32) {
            const imap::SpreadPiece pc = imap::spread_pair_piece(e, CQ, NCOL);
            if (pc.c1 < n1 && pc.c2 < n2 && 2 * pc.j < x3end * NK)
                *reinterpret_cast<float4*>(g0 + pc.s * cstr + pc.c1 * cs1 + pc.c2 * cs2 + 2 * pc.j) =
                    tr[pc.cl * TS + pc.j];
        }
    } else {
        const float2* t2 = reinterpret_cast<const float2*>(tr);
        constexpr int PER = B3 * NK;
        const int tot = ncols * PER;
        for (int e = lane; e < tot; e += 32) {
            const imap::SpreadValue pv = imap::spread_value_piece(e, PER, NK, NCOL);
            if (pv.c1 < n1 && pv.c2 < n2 && pv.x3 < x3end)
                g0[pv.s * cstr + pv.c1 * cs1 + pv.c2 * cs2 + (long long)pv.x3 * nk + pv.q] = t2[pv.cl * TS * 2 + pv.r];
        }
    }
}

// One warp's unit: subproblem `sub` for coils NC * by .. NC * by + NC - 1 (those below B).
template <int B1, int B3, int W, int NK, int NC>
__device__ __forceinline__ void spread_body(const SpreadArgs& a, int kofs, int B, int sub, int by) {
    constexpr int NCOL = B1 * kB2;   // columns of a bin
    constexpr int IPW = 32 / NCOL;   // incidences per warp step
    constexpr int BP = NCOL * B3;
    constexpr int NW = 3 * W;
    static_assert(NCOL * IPW == 32 && B3 % 4 == 0, "bin shape");
    // staging of 32 incidences, reused for the bin's store once they are summed.  Every
    // lane reads each incidence's record (a broadcast, or two with two incidences per
    // step), and a 16-byte shared load costs two L1 wavefronts, so the records are
    // packed: the B3 axis-3 weights as plain floats, and the coefficients
    // conj(V[t, k]) r_b of all NC coils of the warp (the positions and weights of an
    // incidence are staged once and serve every coil) in one run of NCK values, padded
    // to an even count so that it is read 16 bytes at a time.
    constexpr int NCK = NC * NK;
    constexpr int NCKP = (NCK + 1) & ~1;
    constexpr int CQ = imap::spread_cq(B3, NK);
    constexpr int TS = imap::spread_ts(B3, NK);
    constexpr int kStage = 32 * B3 * 4 + 32 * NCKP * 8 + 32 * kNPS * 4;
    constexpr int kTrCols = NC * NCOL > 32 ? NC * NCOL : 32;   // every coil's columns of the bin
    constexpr int kTr = kTrCols * TS * 16;
    using Cls = Axis3Classes<B3, W>;
    __shared__ __align__(16) unsigned char sraw[kStage > kTr ? kStage : kTr];
    float* p3f = reinterpret_cast<float*>(sraw);                 // [incidence][x3]: w3, 0 outside the window
    float2* csm = reinterpret_cast<float2*>(p3f + 32 * B3);      // [incidence][coil][k]: conj(V[t, k]) r_b
    float* psm = reinterpret_cast<float*>(csm + 32 * NCKP);      // [incidence][x1 (B1) | x2 (4) | pad], 0 outside
    float4* tr = reinterpret_cast<float4*>(sraw);
    const Geo& g = a.g;
    const int lane = threadIdx.x;
    const int h = lane / NCOL;   // the lane's incidence slot in a step (0 when B1 = 8)
    const int col = lane % NCOL;
    const int x1 = col >> 2, x2 = col & 3;
    const SubProb sp = a.subs[sub];
    const int b0 = by * NC;                 // first coil of the warp
    const int nc = min(NC, B - b0);         // its coils (the last warp of an odd batch has one)
    const int bin3 = sp.bin % a.nb3;
    const int bt = sp.bin / a.nb3;
    const int bin2 = bt % a.nb2;
    const int bin1 = bt / a.nb2;
    const int lo1 = bin1 * B1, lo2 = bin2 * kB2, lo3 = bin3 * B3;
    const int M1 = g.M[0], M2 = g.M[1], M3 = g.M[2];
    const long long G = (long long)M1 * M2 * M3;
    // a window meets a bin in one contiguous piece along axis 3 when M3 >= B3 + W - 1
    const bool classes = Cls::kOn && M3 >= B3 + W - 1;

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
        int cls = -1;   // the class of staged incidence `lane` (-1: none)
        if (lane < n) {
            const int s = __ldg(a.inc + sp.start + base + lane);
            const float4 p = __ldg(a.pts + s);
            const int orig = __float_as_int(p.w);
            const int t = __ldg(a.tframe + s);
            const float* ws = a.wts + (long long)s * NW;
            // the sample's 3W weights (3W floats from a multiple of 3W: 16-byte loads when
            // 3W is a multiple of 4, 8-byte loads when even)
            float wl[NW];
            if constexpr (NW % 4 == 0) {
#pragma unroll
                for (int q = 0; q < NW; q += 4) {
                    const float4 v = __ldg(reinterpret_cast<const float4*>(ws + q));
                    wl[q] = v.x;
                    wl[q + 1] = v.y;
                    wl[q + 2] = v.z;
                    wl[q + 3] = v.w;
                }
            } else if constexpr (NW % 2 == 0) {
#pragma unroll
                for (int q = 0; q < NW; q += 2) {
                    const float2 v = __ldg(reinterpret_cast<const float2*>(ws + q));
                    wl[q] = v.x;
                    wl[q + 1] = v.y;
                }
            } else {
#pragma unroll
                for (int q = 0; q < NW; ++q) wl[q] = __ldg(ws + q);
            }
            // tap offset of every bin position, wrapped onto the periodic grid:
            // position x takes weight phi_d(a) with a = (lo + x - m0) mod M if a < W
            const int m01 = (int)ceilf(p.x - g.halfW), m02 = (int)ceilf(p.y - g.halfW);
            const int m03 = (int)ceilf(p.z - g.halfW);
            // axis-1 then axis-2 weights, four positions per 16-byte store (positions
            // 4 q .. 4 q + 3 all lie on one axis, as B1 is a multiple of 4)
            float4* pw4 = reinterpret_cast<float4*>(psm + lane * kNPS);
#pragma unroll
            for (int q4 = 0; q4 < (B1 + kB2) / 4; ++q4) {
                const bool ax1 = 4 * q4 < B1;
                const int lo = ax1 ? lo1 : lo2, m0 = ax1 ? m01 : m02, M = ax1 ? M1 : M2, wo = ax1 ? 0 : W;
                const int x0 = ax1 ? 4 * q4 : 4 * q4 - B1;
                float v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    int aa = lo + x0 + u - m0;
                    aa += aa < 0 ? M : 0;
                    aa -= aa >= M ? M : 0;
                    float w = 0.f;
#pragma unroll
                    for (int q = 0; q < W; ++q) w = aa == q ? wl[wo + q] : w;
                    v[u] = w;
                }
                pw4[q4] = make_float4(v[0], v[1], v[2], v[3]);
            }
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
            }
#pragma unroll
            for (int x = 0; x < B3; x += 4)
                *reinterpret_cast<float4*>(p3f + lane * B3 + x) = make_float4(w3v[x], w3v[x + 1], w3v[x + 2], w3v[x + 3]);
            cls = Cls::kAll;
            if (classes) {
                int d = lo3 - m03;   // tap index of bin position 0, wrapped
                d += d < 0 ? M3 : 0;
                d -= d >= M3 ? M3 : 0;
                const int c = (d < W ? -d : M3 - d) + W - 1;
                cls = (c >= 0 && c < Cls::kAll) ? c : Cls::kAll;
            }
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
        // runs of one class (the plan orders a bin's incidences by class; any order is
        // still correct, only slower)
        for (int i = 0; i < n;) {
            const int c = __shfl_sync(kFull, cls, i);
            const unsigned diff = __ballot_sync(kFull, cls != c) & (kFull << i);
            const int e = diff ? __ffs(diff) - 1 : 32;   // lanes >= n hold -1, so e <= n
            spread_class<0, B1, B3, W, NK, NC>(c, acc, psm, p3f, csm, i, e, h, x1, x2);
            i = e;
        }
        __syncwarp();
    }

    if (IPW > 1) {
        // the two half-warps hold sums over alternate incidences of the same columns
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int x3 = 0; x3 < B3; ++x3)
#pragma unroll
                for (int q = 0; q < NK; ++q) {
                    const float2 u = unpack2(acc[c][x3][q]);
                    const float2 v = unpack2(__shfl_xor_sync(kFull, acc[c][x3][q], 16));
                    acc[c][x3][q] = pack2(u.x + v.x, u.y + v.y);
                }
    }

    // store: column (x1, x2) of the bin, element (x3, q) at gbin[x1 cs1 + x2 cs2 + x3 nk + q]
    const int nk = a.nk;
    const long long cs2 = (long long)M3 * nk, cs1 = (long long)M2 * cs2, cstr = G * nk;
    float2* gbin0 = a.grids + (long long)b0 * cstr + (((long long)lo1 * M2 + lo2) * M3 + lo3) * nk + kofs;
    const int n1 = M1 - lo1, n2 = M2 - lo2;
    const int x3end = min(B3, M3 - lo3);
    if (sp.nchunks == 1) {
        // every coil's columns in shared memory at once (column slot c NCOL + col); with two
        // lanes per column (B1 = 4) they write alternate pairs (compile-time indices keep
        // acc in registers)
        __syncwarp();
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int j = 0; j < CQ; ++j)
                if (imap::spread_owns_pair(j, IPW, h))
                    tr[(c * NCOL + col) * TS + j] =
                        pair4(acc[c][(2 * j) / NK][(2 * j) % NK], acc[c][(2 * j + 1) / NK][(2 * j + 1) % NK]);
        __syncwarp();
        store_cols<B1, B3, NK>(tr, nc * NCOL, gbin0, cstr, cs1, cs2, n1, n2, x3end, nk, lane);
        return;
    }
    // multi-chunk bin: the chunk's partial tile of each coil in its slot, 16-byte pair j
    // of column c at [j][c] (each store instruction writes contiguous bytes); with two
    // lanes per column they split the pairs.  The last chunk to arrive (one counter per
    // bin and first coil of the warp) sums them.
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        if (c < nc) {
            float4* part = reinterpret_cast<float4*>(
                a.partials + ((long long)(b0 + c) * a.slots_per_b + sp.slot + sp.chunk) * a.slot_elems +
                (long long)kofs * BP);
#pragma unroll
            for (int j = 0; j < CQ; ++j)
                if (imap::spread_owns_pair(j, IPW, h))
                    part[imap::spread_partial_pair(j, col, NCOL)] =
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
    for (int c0 = 0; c0 < nc; c0 += kTrCols / NCOL) {   // as many coils per pass as shared memory holds
        const int npc = min(kTrCols / NCOL, nc - c0);
        __syncwarp();
        for (int e = lane; e < npc * CQ * NCOL; e += 32) {
            const imap::SpreadPiece pc = imap::spread_sum_piece(e, CQ, NCOL);
            const int c = pc.c, s = pc.s, j = pc.j;
            const float4* part0 = reinterpret_cast<const float4*>(
                a.partials + ((long long)(b0 + c0 + s) * a.slots_per_b + sp.slot) * a.slot_elems +
                (long long)kofs * BP);
            float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int ch = 0; ch < sp.nchunks; ++ch) {
                const float4 v = __ldcg(part0 + ch * slot4 + j * NCOL + c);   // pair j of column c, [j][c]
                sum.x += v.x;
                sum.y += v.y;
                sum.z += v.z;
                sum.w += v.w;
            }
            tr[(s * NCOL + c) * TS + j] = sum;
        }
        __syncwarp();
        store_cols<B1, B3, NK>(tr, npc * NCOL, gbin0 + c0 * cstr, cstr, cs1, cs2, n1, n2, x3end, nk, lane);
    }
    if (lane == 0) *counter = 0;
}

template <int B1, int B3, int W, int NK, int NC>
__global__ void __launch_bounds__(32, NC * B3 * NK <= 20 ? 24 : (NC * B3 * NK <= 40 ? 16 : 1))
spread_kernel(SpreadArgs a, int kofs, int B) {
    spread_body<B1, B3, W, NK, NC>(a, kofs, B, (int)blockIdx.x, (int)blockIdx.y);
}

// Coils per warp: two where the doubled accumulators fit (4-deep columns of at most 5
// channels: 40 packed pairs), else one.
template <int B3, int NK>
__host__ __device__ constexpr int spread_coils() { return spread_pairs_fit(B3, NK) ? 2 : 1; }

template <int B1, int B3, int W, int NK>
cudaError_t launch_wk(const SpreadArgs& a, int kofs, int nsub, int B, int coils, cudaStream_t st) {
    constexpr int NC2 = spread_coils<B3, NK>();
    if (NC2 == 2 && coils != 1 && B >= 2) {
        dim3 grid((unsigned)nsub, (unsigned)((B + 1) / 2));
        spread_kernel<B1, B3, W, NK, NC2><<<grid, 32, 0, st>>>(a, kofs, B);
    } else {
        dim3 grid((unsigned)nsub, (unsigned)B);
        spread_kernel<B1, B3, W, NK, 1><<<grid, 32, 0, st>>>(a, kofs, B);
    }
    return cudaGetLastError();
}

// Channels run in groups of at most 8 (one launch each, exact group size).
template <int B1, int B3, int W>
cudaError_t launch_w(SpreadArgs a, int nsub, int B, int coils, cudaStream_t st) {
    if (a.bs1 != B1 || a.bs2 != kB2 || a.bs3 != B3) return cudaErrorInvalidValue;
    a.ngroups = (a.nk + 7) / 8;
    for (int gi = 0; gi < a.ngroups; ++gi) {
        const int kofs = gi * 8;
        const int ng = a.nk - kofs < 8 ? a.nk - kofs : 8;
        a.group = gi;
        cudaError_t e;
        switch (ng) {
            case 1: e = launch_wk<B1, B3, W, 1>(a, kofs, nsub, B, coils, st); break;
            case 2: e = launch_wk<B1, B3, W, 2>(a, kofs, nsub, B, coils, st); break;
            case 3: e = launch_wk<B1, B3, W, 3>(a, kofs, nsub, B, coils, st); break;
            case 4: e = launch_wk<B1, B3, W, 4>(a, kofs, nsub, B, coils, st); break;
            case 5: e = launch_wk<B1, B3, W, 5>(a, kofs, nsub, B, coils, st); break;
            case 6: e = launch_wk<B1, B3, W, 6>(a, kofs, nsub, B, coils, st); break;
            case 7: e = launch_wk<B1, B3, W, 7>(a, kofs, nsub, B, coils, st); break;
            default: e = launch_wk<B1, B3, W, 8>(a, kofs, nsub, B, coils, st); break;
        }
        if (e != cudaSuccess) return e;
        if (gi > 0) note_launches(1);   // the stage counts its first launch
    }
    return cudaSuccess;
}

template <int B1, int B3>
cudaError_t launch_spread_shape(const Geo& g, const int bs[3], const int nb[3], const SubProb* subs, int nsub,
                                const int* inc, const float4* pts, const int* tframe, const float* wts,
                                const float2* V, const float2* y, const float* scale, int B, int k0, int nk,
                                float2* grids, float2* partials, long long slots_per_b, int* counters, int nbins,
                                int coils, cudaStream_t st) {
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
        case 2: return launch_w<B1, B3, 2>(a, nsub, B, coils, st);
        case 3: return launch_w<B1, B3, 3>(a, nsub, B, coils, st);
        case 4: return launch_w<B1, B3, 4>(a, nsub, B, coils, st);
        case 5: return launch_w<B1, B3, 5>(a, nsub, B, coils, st);
        case 6: return launch_w<B1, B3, 6>(a, nsub, B, coils, st);
        case 7: return launch_w<B1, B3, 7>(a, nsub, B, coils, st);
        case 8: return launch_w<B1, B3, 8>(a, nsub, B, coils, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace
}  // namespace sdp
