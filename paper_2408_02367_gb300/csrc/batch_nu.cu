// Interpolation of several plans in one launch (the batched forward's last
// stage; see batch.cu for the layout of a batched launch and batch_sp.cu for
// the batched spread) for plans that use the row kernel; tiled plans take
// mv_interp_tiles_kernel (interp_tiles.cu).  Kernel widths 4 and 6 only:
// batches of other widths run plan by plan.
#include <algorithm>

#include "batch.cuh"
#include "interp_impl.cuh"

namespace sdp {
namespace {

__device__ __forceinline__ int find_item(const MvUnits& u, long long unit) {
    int i = 0;
    while (i + 1 < u.n && unit >= u.start[i + 1]) ++i;
    return i;
}

// ---- forward: interpolation, persistent warps over the samples of every item ----
// u.start holds the prefix sums of the items' sample counts J.  Warp w takes the
// samples w, w + step, w + 2 step, ... of the concatenated list, walked item by
// item so that an item's pointers and sizes stay loop-invariant over its samples.
// The item loop is unrolled at compile time (up to kMaxMvItems): with a constant
// index, every field of the item is an immediate operand from the launch's
// parameter block, as it is in the single-plan kernel, instead of a register
// loaded per use.
template <int W, int I>
__device__ __forceinline__ void mv_interp_item(const MvArgs& a, const MvUnits& u, const RowLane& rl, long long first,
                                               long long step, int lane) {
    const long long s0 = u.start[I], s1 = u.start[I + 1];
    // this warp's first sample in [s0, s1): the smallest first + k step >= s0
    const long long gs0 = s0 <= first ? first : first + (s0 - first + step - 1) / step * step;
    if (gs0 >= s1) return;
    const MvItem& it = a.it[I];
    const long long J = s1 - s0;
    const long long Gk = (long long)it.g.M[0] * it.g.M[1] * it.g.M[2] * it.g.K;
    for (int b0 = 0; b0 < it.B; b0 += it.interp_coils) {     // one sweep per block of coils
        const int nb = min(it.interp_coils, it.B - b0);
        long long s = gs0 - s0;
        float4 pn = __ldg(it.pts + s);
        int tn = __ldg(it.tframe + s);
        float wn = lane < 3 * W ? __ldg(it.wts + s * (3 * W) + lane) : 0.f;
        for (; s < J; s += step) {
            const float4 p = pn;
            const int t = tn;
            const float wv = wn;
            const long long sn = s + step;
            if (sn < J) {
                pn = __ldg(it.pts + sn);
                tn = __ldg(it.tframe + sn);
                wn = lane < 3 * W ? __ldg(it.wts + sn * (3 * W) + lane) : 0.f;
            }
            interp_rows_sample<W>(it.g, rl, it.V, it.bufA + b0 * Gk, nb, 0, it.g.K, it.y + b0 * J, 0, p, t, wv,
                                  lane);
        }
    }
}

template <int W, int I>
struct MvInterpItems {
    __device__ __forceinline__ static void run(const MvArgs& a, const MvUnits& u, const RowLane& rl, long long first,
                                               long long step, int lane) {
        if (I >= u.n) return;
        mv_interp_item<W, I>(a, u, rl, first, step, lane);
        MvInterpItems<W, I + 1>::run(a, u, rl, first, step, lane);
    }
};
template <int W>
struct MvInterpItems<W, kMaxMvItems> {
    __device__ __forceinline__ static void run(const MvArgs&, const MvUnits&, const RowLane&, long long, long long,
                                               int) {}
};

template <int W, int NT>
__global__ void __launch_bounds__(NT) mv_interp_kernel(const MvArgs a, const MvUnits u) {
    const int lane = threadIdx.x & 31;
    const long long first = ((long long)blockIdx.x * NT + threadIdx.x) >> 5;
    const long long step = ((long long)gridDim.x * NT) >> 5;
    const RowLane rl = row_lane<W>(lane, 0, a.it[0].g.K);   // every item has the same K (one channel group)
    MvInterpItems<W, 0>::run(a, u, rl, first, step, lane);
}

template <int W, int NT>
cudaError_t launch_mv_interp_t(const MvArgs& a, const MvUnits& u, cudaStream_t st) {
    int per_sm = 0, dev = 0, nsm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mv_interp_kernel<W, NT>, NT, 0) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess || nsm < 1)
        return cudaErrorInvalidDevice;
    const long long nres = (long long)nsm * per_sm;
    const long long nneed = (u.start[u.n] + NT / 32 - 1) / (NT / 32);
    mv_interp_kernel<W, NT><<<(unsigned)std::min(nneed, nres), NT, 0, st>>>(a, u);
    return cudaGetLastError();
}

template <int W>
cudaError_t launch_mv_interp_w(const MvArgs& a, const MvUnits& u, int threads, cudaStream_t st) {
    if (W <= 4 && threads == 1024) return launch_mv_interp_t<W, (W <= 4 ? 1024 : 256)>(a, u, st);
    return launch_mv_interp_t<W, 256>(a, u, st);
}

}  // namespace

bool mv_width_supported(int W) { return W == 4 || W == 6; }

cudaError_t launch_mv_interp(const MvArgs& a, const MvUnits& u, int W, int threads, cudaStream_t st) {
    if (u.start[u.n] == 0) return cudaSuccess;
    switch (W) {
        case 4: return launch_mv_interp_w<4>(a, u, threads, st);
        case 6: return launch_mv_interp_w<6>(a, u, threads, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sdp
