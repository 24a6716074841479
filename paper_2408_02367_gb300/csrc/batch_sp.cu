// Spread of several plans in one launch (the batched adjoint's first stage; see
// batch.cu for the layout of a batched launch).  One warp per (subproblem, coil
// pair or coil) of every item, running the single-plan spread's body
// (spread_impl.cuh) on that item's plan.  Kernel widths 4 and 6, one channel
// group (K <= 32 / W), items of one bin shape.
#include "batch.cuh"
#include "spread_impl.cuh"

namespace sdp {
namespace {

__device__ __forceinline__ int find_item(const MvUnits& u, long long unit) {
    int i = 0;
    while (i + 1 < u.n && unit >= u.start[i + 1]) ++i;
    return i;
}

// u.start holds the prefix sums of nsub * (coil groups) per item.
template <int B1, int B3, int W, int NK>
__global__ void __launch_bounds__(32, 16) mv_spread_kernel(const MvArgs a, const MvUnits u) {
    const long long unit = blockIdx.x;
    const int i = find_item(u, unit);
    const MvItem& it = a.it[i];
    const long long local = unit - u.start[i];
    const int sub = (int)(local % it.nsub);
    const int by = (int)(local / it.nsub);
    constexpr int NC2 = spread_coils<B3, NK>();
    if (NC2 == 2 && it.spread_pairs)
        spread_body<B1, B3, W, NK, NC2>(it.sa, 0, it.B, sub, by);
    else
        spread_body<B1, B3, W, NK, 1>(it.sa, 0, it.B, sub, by);
}

// One channel group of at most 32 / W channels (the batched path's eligibility).
template <int B1, int B3, int W, int NK>
cudaError_t launch_mv_spread_k(const MvArgs& a, const MvUnits& u, cudaStream_t st) {
    if constexpr (NK <= 32 / W) {
        mv_spread_kernel<B1, B3, W, NK><<<(unsigned)u.start[u.n], 32, 0, st>>>(a, u);
        return cudaGetLastError();
    } else {
        return cudaErrorInvalidValue;
    }
}

template <int B1, int B3, int W>
cudaError_t launch_mv_spread_w(const MvArgs& a, const MvUnits& u, int K, cudaStream_t st) {
    switch (K) {
        case 1: return launch_mv_spread_k<B1, B3, W, 1>(a, u, st);
        case 2: return launch_mv_spread_k<B1, B3, W, 2>(a, u, st);
        case 3: return launch_mv_spread_k<B1, B3, W, 3>(a, u, st);
        case 4: return launch_mv_spread_k<B1, B3, W, 4>(a, u, st);
        case 5: return launch_mv_spread_k<B1, B3, W, 5>(a, u, st);
        case 6: return launch_mv_spread_k<B1, B3, W, 6>(a, u, st);
        case 7: return launch_mv_spread_k<B1, B3, W, 7>(a, u, st);
        case 8: return launch_mv_spread_k<B1, B3, W, 8>(a, u, st);
        default: return cudaErrorInvalidValue;
    }
}

template <int B1, int B3>
cudaError_t launch_mv_spread_b(const MvArgs& a, const MvUnits& u, int W, int K, cudaStream_t st) {
    switch (W) {
        case 4: return launch_mv_spread_w<B1, B3, 4>(a, u, K, st);
        case 6: return launch_mv_spread_w<B1, B3, 6>(a, u, K, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_mv_spread(const MvArgs& a, const MvUnits& u, int bin_width, int bin_depth, int W, int K,
                             cudaStream_t st) {
    if (u.start[u.n] == 0) return cudaSuccess;
    if (u.start[u.n] > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    if (bin_width == 4)
        return bin_depth == 4 ? launch_mv_spread_b<4, 4>(a, u, W, K, st) : launch_mv_spread_b<4, 8>(a, u, W, K, st);
    return bin_depth == 4 ? launch_mv_spread_b<8, 4>(a, u, W, K, st) : launch_mv_spread_b<8, 8>(a, u, W, K, st);
}

}  // namespace sdp
