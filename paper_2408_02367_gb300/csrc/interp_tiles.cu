// Forward interpolation with the subspace contraction (gridding step A3, the
// same operation as interp.cu), from shared-memory tiles:
//
//   y_b[j] = sum_k V[t_j, k] sum_{W^3 taps} phi(g1 - m1) phi(g2 - m2) phi(g3 - m3) U_{b,k}[m mod M]
//
// for the per-coil operator A_c of StoDIP (Sec. 2 Eq. 1, Sec. 2.1 Eq. 3).
//
// The plan orders the samples by tile of 8 x 8 x 8 grid points (the tile of
// the sample's own coordinate) and lists work items, heaviest first: each
// non-empty tile, a dense one cut into pieces of at most 512 samples (the
// k-space centre's tiles hold thousands, which one CTA would serialise).
// A sample of tile t has its window start m0 = ceil(g - W/2) in
// [8 t - W/2, 8 t + 8 - W/2] along each axis, so its W^3 taps lie in the
// (8 + W)^3 points from 8 t - W/2.  Persistent CTAs walk the work items; for each
// coil a CTA copies those points x nk channels of the channel-interleaved grid
// ([b][i1][i2][i3][kk], wrapped periodically) into shared memory: one bulk copy
// (cp.async.bulk) per row, two where the row wraps around the grid along axis 3,
// completing on an mbarrier whose wait is bounded (W = 4; for W = 2 rows that do
// not start on a 16-byte boundary, cp.async 8 bytes per value), and then
// interpolates every sample of the item from shared memory.  The scattered,
// latency-bound gathers of the row kernel become one coalesced copy per tile
// and coil plus shared loads.
//
// A warp takes two samples at a time, one per half-warp.  Lane (a2, a3) of a
// half-warp (W^2 <= 16 lanes) owns the axis-2/axis-3 tap pair: over the W
// axis-1 taps it accumulates phi1(a1) U_k for its tap's nk channels (shared
// loads at compile-time offsets from one base address), contracts them with
// V[t, k], scales by phi2(a2) phi3(a3), and the half-warp sums its lanes.  The
// next pair's coordinates, frame and weights are loaded while the current pair
// is interpolated.
// Widths 2 and 4, up to 8 channels per call; other calls use interp.cu.
#include <atomic>

#include "batch.cuh"
#include "index_map.cuh"
#include "interp_impl.cuh"
#include "tma.cuh"

namespace sdp {
namespace {

constexpr int kTile = 8;              // tile edge in grid points (the plan's sample order)
constexpr int kTileThreads = 256;

__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <int W, int NK>
struct TileDims {
    static constexpr int H = kTile + W;   // tile plus window margin, per axis
    static constexpr int ROW = H * NK;    // complex values of one (h1, h2) row
    static constexpr int PLANE = H * ROW;
    static constexpr int SIZE = H * PLANE;
    static constexpr int BYTES = SIZE * 8;
    static constexpr int SMEM = BYTES + 16;   // the tile and the copies' mbarrier
};

// One work item td = (flattened tile index, first sample, sample count, -): for each
// coil the item's tile is copied into sg (bulk copies completing on bar, or cp.async),
// then the item's samples are interpolated from it.  False if a copy did not land
// within the wait's bound (status then holds SDP_ERR_TIMEOUT and the caller leaves).
template <int W, int NK, bool TEST = false>
__device__ __forceinline__ bool tile_work(const Geo& g, const int4 td, int nt2, int nt3,
                                          const float4* __restrict__ pts, const int* __restrict__ tframe,
                                          const float* __restrict__ wts, const float2* __restrict__ V,
                                          const float2* __restrict__ grids, int B, int k0, float2* __restrict__ y,
                                          int accumulate, int* status, float2* sg, uint64_t* bar, uint32_t& phase,
                                          int withhold_row, unsigned long long wait_ns) {
    using D = TileDims<W, NK>;
    constexpr int H = D::H, ROW = D::ROW, PLANE = D::PLANE;
    constexpr int NWARP = kTileThreads / 32;
    constexpr int HW = W / 2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int half = lane >> 4, l16 = lane & 15;
    const imap::TileLane tl = imap::tile_lane_map(l16, W);   // idle lanes repeat tap (0, 0) with zero weight
    const bool act = tl.act;
    const int a2 = tl.a2, a3 = tl.a3;
    const int M1 = g.M[0], M2 = g.M[1], M3 = g.M[2];
    const long long Gk = (long long)M1 * M2 * M3 * NK;
    const long long J = g.J;
    const int t3 = td.x % nt3, t12 = td.x / nt3;
    const int t2 = t12 % nt2, t1 = t12 / nt2;
    const int lo1 = t1 * kTile - HW, lo2 = t2 * kTile - HW, lo3 = t3 * kTile - HW;
    const int start = td.y, count = td.z;
    // a row's H points along axis 3 start at p0 and run la points before they wrap
    // around the grid (la = H unless the tile crosses the grid's end along axis 3)
    const int p0 = wrap1(lo3, M3);
    const int la = M3 - p0 < H ? M3 - p0 : H;
    for (int b = 0; b < B; ++b) {
        __syncthreads();   // the previous pass's readers are done with sg
        const float2* gb = grids + (long long)b * Gk;
        // Bulk copies, one per row piece (one or two pieces per row), where every
        // piece starts on a 16-byte boundary (p0 NK and la NK even, the grid aligned:
        // W = 4 tiles always); else cp.async 8 bytes per value.
        const bool bulk = ((p0 * NK) & 1) == 0 && ((la * NK) & 1) == 0 &&
                          (reinterpret_cast<unsigned long long>(gb) & 15) == 0;
        if (bulk) {
            if (threadIdx.x == 0) tma::mbar_expect_tx(bar, (uint32_t)D::BYTES);
            __syncthreads();   // the expected bytes are registered before any copy lands
            for (int r = threadIdx.x; r < H * H; r += kTileThreads) {
                if (TEST && b == 0 && r == withhold_row) continue;   // the wait test hook: this row never lands
                const int h1 = r / H, h2 = r - h1 * H;
                const float2* src = gb + ((long long)wrap1(lo1 + h1, M1) * M2 + wrap1(lo2 + h2, M2)) * M3 * NK;
                float2* dst = sg + r * ROW;
                tma::bulk_g2s(dst, src + (long long)p0 * NK, (uint32_t)(la * NK * 8), bar);
                if (la < H) tma::bulk_g2s(dst + la * NK, src, (uint32_t)((H - la) * NK * 8), bar);
            }
            const bool landed =
                __syncthreads_and(tma::mbar_wait(bar, phase, status, TEST ? wait_ns : tma::kWaitNs)) != 0;
            if (!landed) {
                // a copy did not complete within the wait's bound (status holds
                // SDP_ERR_TIMEOUT): give the copies in flight one more bounded wait, leave
                tma::mbar_wait(bar, phase, nullptr, TEST ? wait_ns : tma::kWaitNs);
                return false;
            }
            phase ^= 1u;
        } else {
            for (int r = warp; r < H * H; r += NWARP) {
                const int h1 = r / H, h2 = r - h1 * H;
                const float2* src = gb + ((long long)wrap1(lo1 + h1, M1) * M2 + wrap1(lo2 + h2, M2)) * M3 * NK;
                float2* dst = sg + r * ROW;
                for (int c = lane; c < ROW; c += 32) {
                    const int h3 = c / NK, k = c - h3 * NK;
                    cp_async8(dst + c, src + wrap1(lo3 + h3, M3) * NK + k);
                }
            }
            cp_async_wait_all();
            __syncthreads();
        }
        // a warp takes the sample pairs q = warp, warp + NWARP, ...; the next pair's
        // coordinates, frame and weights are loaded while the current pair is interpolated
        auto fetch = [&](int qq, float4& p, int& t, float (&w1)[W], float& w23) {
            const int si = 2 * qq + half;
            const long long s = start + (si < count ? si : 2 * qq);   // a second half without a sample repeats the first
            p = __ldg(pts + s);
            t = __ldg(tframe + s);
            const float* ws = wts + s * (3 * W);
            if constexpr (W == 4) {   // 48 bytes per sample: the axis-1 weights are one aligned 16-byte load
                const float4 v = __ldg(reinterpret_cast<const float4*>(ws));
                w1[0] = v.x;
                w1[1] = v.y;
                w1[2] = v.z;
                w1[3] = v.w;
            } else {
#pragma unroll
                for (int a = 0; a < W; ++a) w1[a] = __ldg(ws + a);
            }
            w23 = __ldg(ws + W + a2) * __ldg(ws + 2 * W + a3);
        };
        float4 pn = make_float4(0.f, 0.f, 0.f, 0.f);
        int tn = 0;
        float w1n[W], w23n = 0.f;
        if (2 * warp < count) fetch(warp, pn, tn, w1n, w23n);
        for (int q = warp; 2 * q < count; q += NWARP) {
            const bool ok = 2 * q + half < count;
            const float4 p = pn;
            const int t = tn;
            float w1[W];
#pragma unroll
            for (int a = 0; a < W; ++a) w1[a] = w1n[a];
            float w23 = w23n;
            if (2 * (q + NWARP) < count) fetch(q + NWARP, pn, tn, w1n, w23n);
            const float2* Vt = V + (long long)t * g.K + k0;
            float2 vk[NK];
#pragma unroll
            for (int k = 0; k < NK; ++k) vk[k] = __ldg(Vt + k);
            const int orig = __float_as_int(p.w);
            const int d1 = (int)ceilf(p.x - g.halfW) - lo1;
            const int d2 = (int)ceilf(p.y - g.halfW) - lo2;
            const int d3 = (int)ceilf(p.z - g.halfW) - lo3;
            // the window lies in the tile by construction of the plan's order; a sample
            // outside it would read the wrong points, so it is reported and contributes 0
            const bool inside = (unsigned)d1 <= kTile && (unsigned)d2 <= kTile && (unsigned)d3 <= kTile;
            const int e1 = inside ? d1 : 0, e2 = inside ? d2 : 0, e3 = inside ? d3 : 0;
            w23 = (act && ok && inside) ? w23 : 0.f;
            const unsigned long long* base =
                reinterpret_cast<const unsigned long long*>(sg + imap::tile_offset(e1, e2, e3, 0, a2, a3, 0, H, NK));
            unsigned long long acc[NK];
#pragma unroll
            for (int k = 0; k < NK; ++k) acc[k] = 0ull;
#pragma unroll
            for (int a1 = 0; a1 < W; ++a1) {
                const unsigned long long wa = pk2(w1[a1], w1[a1]);
#pragma unroll
                for (int k = 0; k < NK; ++k) acc[k] = fma2(wa, base[a1 * PLANE + k], acc[k]);
            }
            float sx = 0.f, sy = 0.f;
#pragma unroll
            for (int k = 0; k < NK; ++k) {
                const float2 v = vk[k];
                const float2 u = upk2(acc[k]);
                sx = fmaf(v.x, u.x, sx);
                sx = fmaf(-v.y, u.y, sx);
                sy = fmaf(v.x, u.y, sy);
                sy = fmaf(v.y, u.x, sy);
            }
            sx *= w23;
            sy *= w23;
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) {
                sx += __shfl_xor_sync(kFullI, sx, o);
                sy += __shfl_xor_sync(kFullI, sy, o);
            }
            if (ok && l16 == 0) {
                if (inside)
                    put(y + (long long)b * J + orig, sx, sy, accumulate);
                else
                    atomicCAS(status, 0, SDP_ERR_BOUNDS);
            }
        }
    }
    return true;
}

// TEST: the instantiation that honours the wait test hook (withhold_row, wait_ns);
// the other ignores both, so the hook costs the production kernel nothing.
template <int W, int NK, bool TEST>
__global__ void __launch_bounds__(kTileThreads) interp_tiles_kernel(Geo g, const int4* __restrict__ tiles, int ntiles,
                                                                    int nt2, int nt3, const float4* __restrict__ pts,
                                                                    const int* __restrict__ tframe,
                                                                    const float* __restrict__ wts,
                                                                    const float2* __restrict__ V,
                                                                    const float2* __restrict__ grids, int B, int k0,
                                                                    float2* __restrict__ y, int accumulate,
                                                                    int* status, int withhold_row,
                                                                    unsigned long long wait_ns) {
    using D = TileDims<W, NK>;
    static_assert(D::ROW % 2 == 0 && D::SIZE % 2 == 0, "16-byte row pieces, 8-byte aligned mbarrier");
    extern __shared__ __align__(16) float2 sg[];   // [h1][h2][h3][k], then the copies' mbarrier
    uint64_t* bar = reinterpret_cast<uint64_t*>(sg + D::SIZE);
    if (threadIdx.x == 0) {
        tma::mbar_init(bar, 1);
        tma::fence_init();
    }
    __syncthreads();
    uint32_t phase = 0;
    for (int it = blockIdx.x; it < ntiles; it += gridDim.x)
        if (!tile_work<W, NK, TEST>(g, tiles[it], nt2, nt3, pts, tframe, wts, V, grids, B, k0, y, accumulate, status,
                                    sg, bar, phase, it == 0 ? withhold_row : -1, wait_ns))
            return;
}

// Several plans in one launch (the batched forward's interpolation): the work
// items of every item of the batch, u.start holding the prefix sums of the items'
// work-item counts; each work item runs the single-plan body on its item's plan.
__device__ __forceinline__ int mv_find_item(const MvUnits& u, long long unit) {
    int i = 0;
    while (i + 1 < u.n && unit >= u.start[i + 1]) ++i;
    return i;
}

template <int W, int NK>
__global__ void __launch_bounds__(kTileThreads) mv_interp_tiles_kernel(const MvArgs a, const MvUnits u) {
    using D = TileDims<W, NK>;
    extern __shared__ __align__(16) float2 sg[];   // [h1][h2][h3][k], then the copies' mbarrier
    uint64_t* bar = reinterpret_cast<uint64_t*>(sg + D::SIZE);
    if (threadIdx.x == 0) {
        tma::mbar_init(bar, 1);
        tma::fence_init();
    }
    __syncthreads();
    uint32_t phase = 0;
    for (long long w = blockIdx.x; w < u.start[u.n]; w += gridDim.x) {
        const int i = mv_find_item(u, w);
        const MvItem& it = a.it[i];
        if (!tile_work<W, NK>(it.g, it.itiles[w - u.start[i]], it.nt2, it.nt3, it.pts, it.tframe, it.wts, it.V,
                              it.bufA, it.B, 0, it.y, 0, it.status, sg, bar, phase, -1, tma::kWaitNs))
            return;
    }
}

// Resident CTAs per SM of a tiled kernel, found once per instantiation.
template <class K>
cudaError_t tiles_grid(K kernel, int bytes, long long nwork, std::atomic<int>& resident, unsigned& grid) {
    int per_sm = resident.load(std::memory_order_relaxed);
    if (per_sm == 0) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kTileThreads, bytes);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) per_sm = 1;
        resident.store(per_sm, std::memory_order_relaxed);
    }
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess || nsm < 1)
        return cudaErrorInvalidDevice;
    const long long nres = (long long)nsm * per_sm;
    grid = (unsigned)(nwork < nres ? nwork : nres);
    return cudaSuccess;
}

template <int W, int NK>
cudaError_t launch_mv_tiles_k(const MvArgs& a, const MvUnits& u, cudaStream_t st) {
    constexpr int bytes = TileDims<W, NK>::SMEM;
    static std::atomic<int> resident{0};
    unsigned grid = 0;
    const cudaError_t e = tiles_grid(mv_interp_tiles_kernel<W, NK>, bytes, u.start[u.n], resident, grid);
    if (e != cudaSuccess) return e;
    mv_interp_tiles_kernel<W, NK><<<grid, kTileThreads, bytes, st>>>(a, u);
    return cudaGetLastError();
}

template <int W>
cudaError_t launch_mv_tiles_w(const MvArgs& a, const MvUnits& u, int K, cudaStream_t st) {
    switch (K) {
        case 1: return launch_mv_tiles_k<W, 1>(a, u, st);
        case 2: return launch_mv_tiles_k<W, 2>(a, u, st);
        case 3: return launch_mv_tiles_k<W, 3>(a, u, st);
        case 4: return launch_mv_tiles_k<W, 4>(a, u, st);
        case 5: return launch_mv_tiles_k<W, 5>(a, u, st);
        case 6: return launch_mv_tiles_k<W, 6>(a, u, st);
        case 7: return launch_mv_tiles_k<W, 7>(a, u, st);
        case 8: return launch_mv_tiles_k<W, 8>(a, u, st);
        default: return cudaErrorInvalidValue;
    }
}

template <int W, int NK>
cudaError_t launch_tiles_k(const Geo& g, const int4* tiles, int ntiles, int nt2, int nt3, const float4* pts,
                           const int* tframe, const float* wts, const float2* V, const float2* grids, int B, int k0,
                           float2* y, int accumulate, int* status, int withhold_row, unsigned long long wait_ns,
                           cudaStream_t st) {
    constexpr int bytes = TileDims<W, NK>::SMEM;
    static std::atomic<int> resident{0};
    unsigned grid = 0;
    const bool test = withhold_row >= 0 || wait_ns != tma::kWaitNs;
    const cudaError_t e = tiles_grid(interp_tiles_kernel<W, NK, false>, bytes, ntiles, resident, grid);
    if (e != cudaSuccess) return e;
    if (test) {
        static std::atomic<int> resident_t{0};
        unsigned grid_t = 0;
        const cudaError_t et = tiles_grid(interp_tiles_kernel<W, NK, true>, bytes, ntiles, resident_t, grid_t);
        if (et != cudaSuccess) return et;
        interp_tiles_kernel<W, NK, true><<<grid_t, kTileThreads, bytes, st>>>(
            g, tiles, ntiles, nt2, nt3, pts, tframe, wts, V, grids, B, k0, y, accumulate, status, withhold_row, wait_ns);
    } else {
        interp_tiles_kernel<W, NK, false><<<grid, kTileThreads, bytes, st>>>(
            g, tiles, ntiles, nt2, nt3, pts, tframe, wts, V, grids, B, k0, y, accumulate, status, -1, tma::kWaitNs);
    }
    return cudaGetLastError();
}

template <int W>
cudaError_t launch_tiles_w(const Geo& g, const int4* tiles, int ntiles, int nt2, int nt3, const float4* pts,
                           const int* tframe, const float* wts, const float2* V, const float2* grids, int B, int k0,
                           int nk, float2* y, int accumulate, int* status, int wr, unsigned long long wn,
                           cudaStream_t st) {
    switch (nk) {
        case 1: return launch_tiles_k<W, 1>(g, tiles, ntiles, nt2, nt3, pts, tframe, wts, V, grids, B, k0, y, accumulate, status, wr, wn, st);
        case 2: return launch_tiles_k<W, 2>(g, tiles, ntiles, nt2, nt3, pts, tframe, wts, V, grids, B, k0, y, accumulate, status, wr, wn, st);
        case 3: return launch_tiles_k<W, 3>(g, tiles, ntiles, nt2, nt3, pts, tframe, wts, V, grids, B, k0, y, accumulate, status, wr, wn, st);
        case 4: return launch_tiles_k<W, 4>(g, tiles, ntiles, nt2, nt3, pts, tframe, wts, V, grids, B, k0, y, accumulate, status, wr, wn, st);
        case 5: return launch_tiles_k<W, 5>(g, tiles, ntiles, nt2, nt3, pts, tframe, wts, V, grids, B, k0, y, accumulate, status, wr, wn, st);
        case 6: return launch_tiles_k<W, 6>(g, tiles, ntiles, nt2, nt3, pts, tframe, wts, V, grids, B, k0, y, accumulate, status, wr, wn, st);
        case 7: return launch_tiles_k<W, 7>(g, tiles, ntiles, nt2, nt3, pts, tframe, wts, V, grids, B, k0, y, accumulate, status, wr, wn, st);
        case 8: return launch_tiles_k<W, 8>(g, tiles, ntiles, nt2, nt3, pts, tframe, wts, V, grids, B, k0, y, accumulate, status, wr, wn, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

int interp_tile_edge() { return kTile; }

bool interp_tiles_supported(int W, int nk) { return (W == 2 || W == 4) && nk >= 1 && nk <= 8; }

cudaError_t launch_mv_interp_tiles(const MvArgs& a, const MvUnits& u, int W, int K, cudaStream_t st) {
    if (u.start[u.n] == 0) return cudaSuccess;
    switch (W) {
        case 2: return launch_mv_tiles_w<2>(a, u, K, st);
        case 4: return launch_mv_tiles_w<4>(a, u, K, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_interp_tiles(const Geo& g, const int4* tiles, int ntiles, int nt2, int nt3, const float4* pts,
                                const int* tframe, const float* wts, const float2* V, const float2* grids, int B,
                                int k0, int nk, float2* y, int accumulate, int* status, int withhold_row,
                                long long wait_ns, cudaStream_t st) {
    const int wr = withhold_row;
    const unsigned long long wn = wait_ns > 0 ? (unsigned long long)wait_ns : tma::kWaitNs;
    if (ntiles == 0 || B == 0) return cudaSuccess;
    switch (g.W) {
        case 2: return launch_tiles_w<2>(g, tiles, ntiles, nt2, nt3, pts, tframe, wts, V, grids, B, k0, nk, y, accumulate, status, wr, wn, st);
        case 4: return launch_tiles_w<4>(g, tiles, ntiles, nt2, nt3, pts, tframe, wts, V, grids, B, k0, nk, y, accumulate, status, wr, wn, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sdp
