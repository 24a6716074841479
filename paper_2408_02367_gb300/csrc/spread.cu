// Adjoint spreading, bins of 8 x 4 x 8 grid points, and the bin-shape dispatch
// of launch_spread (the kernel itself is in spread_impl.cuh; spread_b4.cu
// instantiates the 8 x 4 x 4 bins in a translation unit of its own).
#include "spread_impl.cuh"

namespace sdp {

cudaError_t launch_spread_b4(const Geo& g, const int bs[3], const int nb[3], const SubProb* subs, int nsub,
                             const int* inc, const float4* pts, const int* tframe, const float* wts, const float2* V,
                             const float2* y, const float* scale, int B, int k0, int nk, float2* grids,
                             float2* partials, long long slots_per_b, int* counters, int nbins, int coils,
                             cudaStream_t st);

bool spread_bins_supported(const int bs[3]) { return bs[0] == 8 && bs[1] == 4 && (bs[2] == 8 || bs[2] == 4); }

cudaError_t launch_spread(const Geo& g, const int bs[3], const int nb[3], const SubProb* subs, int nsub,
                          const int* inc, const float4* pts, const int* tframe, const float* wts, const float2* V,
                          const float2* y, const float* scale, int B, int k0, int nk, float2* grids,
                          float2* partials, long long slots_per_b, int* counters, int nbins, int coils,
                          cudaStream_t st) {
    if (bs[2] == 4)
        return launch_spread_b4(g, bs, nb, subs, nsub, inc, pts, tframe, wts, V, y, scale, B, k0, nk, grids, partials,
                                slots_per_b, counters, nbins, coils, st);
    return launch_spread_depth<8>(g, bs, nb, subs, nsub, inc, pts, tframe, wts, V, y, scale, B, k0, nk, grids,
                                  partials, slots_per_b, counters, nbins, coils, st);
}

}  // namespace sdp
