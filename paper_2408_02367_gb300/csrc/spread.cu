// Adjoint spreading: the bin-shape dispatch of launch_spread and the bins of
// 8 x 4 x 8 grid points.  The kernel itself is in spread_impl.cuh; each other bin
// shape is instantiated in a translation unit of its own (spread_b4.cu: 8 x 4 x 4,
// spread_4x4x8.cu and spread_4x4x4.cu: two incidences per warp step).
#include "spread_impl.cuh"

namespace sdp {

#define SDP_SPREAD_SHAPE_DECL(name)                                                                                   \
    cudaError_t name(const Geo& g, const int bs[3], const int nb[3], const SubProb* subs, int nsub, const int* inc, \
                     const float4* pts, const int* tframe, const float* wts, const float2* V, const float2* y,      \
                     const float* scale, int B, int k0, int nk, float2* grids, float2* partials,                   \
                     long long slots_per_b, int* counters, int nbins, int coils, cudaStream_t st)
SDP_SPREAD_SHAPE_DECL(launch_spread_b4);
SDP_SPREAD_SHAPE_DECL(launch_spread_448);
SDP_SPREAD_SHAPE_DECL(launch_spread_444);
#undef SDP_SPREAD_SHAPE_DECL

bool spread_bins_supported(const int bs[3]) {
    return (bs[0] == 8 || bs[0] == 4) && bs[1] == 4 && (bs[2] == 8 || bs[2] == 4);
}

cudaError_t launch_spread(const Geo& g, const int bs[3], const int nb[3], const SubProb* subs, int nsub,
                          const int* inc, const float4* pts, const int* tframe, const float* wts, const float2* V,
                          const float2* y, const float* scale, int B, int k0, int nk, float2* grids,
                          float2* partials, long long slots_per_b, int* counters, int nbins, int coils,
                          cudaStream_t st) {
    if (!spread_bins_supported(bs)) return cudaErrorInvalidValue;
    auto fn = bs[0] == 8 ? (bs[2] == 4 ? launch_spread_b4 : launch_spread_shape<8, 8>)
                         : (bs[2] == 4 ? launch_spread_444 : launch_spread_448);
    return fn(g, bs, nb, subs, nsub, inc, pts, tframe, wts, V, y, scale, B, k0, nk, grids, partials, slots_per_b,
              counters, nbins, coils, st);
}

}  // namespace sdp
