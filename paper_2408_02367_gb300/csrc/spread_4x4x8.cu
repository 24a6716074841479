// Adjoint spreading with bins of 4 x 4 x 8 grid points: 16 columns, two
// incidences per warp step (one per half-warp).
// The kernel is in spread_impl.cuh.
#include "spread_impl.cuh"

namespace sdp {

cudaError_t launch_spread_448(const Geo& g, const int bs[3], const int nb[3], const SubProb* subs, int nsub,
                              const int* inc, const float4* pts, const int* tframe, const float* wts, const float2* V,
                              const float2* y, const float* scale, int B, int k0, int nk, float2* grids,
                              float2* partials, long long slots_per_b, int* counters, int nbins, int coils,
                              cudaStream_t st) {
    return launch_spread_shape<4, 8>(g, bs, nb, subs, nsub, inc, pts, tframe, wts, V, y, scale, B, k0, nk, grids,
                                      partials, slots_per_b, counters, nbins, coils, st);
}

}  // namespace sdp
