// Internal definitions shared by the kernels and the C ABI of the subspace
// multicoil NUFFT operator.  Not part of the public interface.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/stodip_op.h"

namespace sdp {

constexpr int kMaxRadixStages = 12;
constexpr int kMaxWidth = 8;
constexpr int kMaxK = 16;
constexpr int kMaxBatch = 64;
constexpr int kNumStages = 10;  // profiling stages, see stodip_op.h

enum Stage {
    ST_FWD_FFT3 = 0,
    ST_FWD_FFT2 = 1,
    ST_FWD_FFT1 = 2,
    ST_INTERP = 3,
    ST_SPREAD = 4,
    ST_ADJ_FFT1 = 5,
    ST_ADJ_FFT2 = 6,
    ST_ADJ_FFT3 = 7,
    ST_LOSS = 8,
    ST_TV = 9,
};

// One axis of the 3D FFT: length L = prod(radix[0..nst)), twiddles
// tw[m] = exp(-2 pi i m / L) in float32 (computed in float64 on the host).
struct FftAxis {
    int L;
    int nst;
    int radix[kMaxRadixStages];
    const float2* tw;
    int generic;   // 1: always the Stockham kernels (a plan's tuning), 0: two-pass where available
    int lines;     // lines per CTA of the fused axis-3 kernels: 0 = default, 8 or 4
    int cols;      // columns per CTA of the strided axis-1/axis-2 passes: 0 = default, 32 or 8
    int staged;    // fused axis-3 kernels staged by bulk copies where supported: bit 0 prologue, bit 1 epilogue
};

// A spread subproblem: one chunk of the incidence list of one output bin.
struct SubProb {
    int bin;       // flattened bin index
    int start;     // first incidence
    int count;     // incidences in this chunk
    int chunk;     // chunk number within the bin
    int nchunks;   // chunks of this bin (1 = write the bin directly)
    int slot;      // partial-tile slot of chunk 0 of this bin (multi-chunk bins)
};

// Shared view of a plan passed to the kernel launchers.
struct Geo {
    int N[3];
    int M[3];
    int W;
    int K;
    int T;
    int C;
    int J;
    float beta;
    float inv_i0_beta;
    float halfW;
};

// Arguments of the spread kernels (spread_impl.cuh) for one plan and call.
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
    int ngroups;   // channel groups of this call (counters are per group)
    int group;
};

// Whether one spread warp can hold the register columns of two coils (bins of depth
// B3, NK channels in the group): 40 packed accumulator pairs at most.
__host__ __device__ constexpr bool spread_pairs_fit(int B3, int NK) { return B3 * NK <= 20; }

// Launch helpers (each returns cudaError_t of the launch).  `pr` may be null.
// Spread bin shapes with a kernel: B1 x 4 x B3 grid points, B1 and B3 each 8 or 4.
bool spread_bins_supported(const int bs[3]);
cudaError_t launch_fwd_prologue_fft3(const Geo& g, const FftAxis& ax, const float2* x, const float2* S,
                                     const int* coil_idx, int B, int k0, int nk, const float* dinv1,
                                     const float* dinv2, const float* dinv3, float2* out, int* status,
                                     cudaStream_t st);
cudaError_t launch_fft_strided(const FftAxis& ax, int inverse, const float2* in, float2* out, int n_in,
                               int in_centred, int n_out, int out_centred, long long inner, long long outer,
                               cudaStream_t st);
cudaError_t launch_adj_fft3_epilogue(const Geo& g, const FftAxis& ax, const float2* in, const float2* S,
                                     const int* coil_idx, int B, int k0, int nk, const float* dinv1,
                                     const float* dinv2, const float* dinv3, float2* out, int accumulate,
                                     int* status, cudaStream_t st);
// Kaiser-Bessel weights of every (sorted) sample: wts[s][d][a] = phi(g_d - (m0_d + a)),
// m0_d = ceil(g_d - W/2) in float32; computed once per plan.
cudaError_t launch_kb_weights(const Geo& g, const float4* pts, float* wts, cudaStream_t st);
// Tiled interpolation (interp_tiles.cu): samples ordered by tiles of
// interp_tile_edge()^3 grid points; `tiles` lists work items (flattened tile
// index over nt1 x nt2 x nt3, first sample, count, 0), a dense tile's samples
// split over several items.
int interp_tile_edge();
bool interp_tiles_supported(int W, int nk);
cudaError_t launch_interp_tiles(const Geo& g, const int4* tiles, int ntiles, int nt2, int nt3, const float4* pts,
                                const int* tframe, const float* wts, const float2* V, const float2* grids, int B,
                                int k0, int nk, float2* y, int accumulate, int* status, int withhold_row,
                                long long wait_ns, cudaStream_t st);
cudaError_t launch_interp(const Geo& g, int threads, int run, int cblock, const float4* pts, const int* tframe,
                          const float* wts,
                          const float2* V, const float2* grids, int B, int k0, int nk, float2* y, int accumulate,
                          cudaStream_t st);
cudaError_t launch_spread(const Geo& g, const int bs[3], const int nb[3], const SubProb* subs, int nsub,
                          const int* inc, const float4* pts, const int* tframe, const float* wts, const float2* V,
                          const float2* y, const float* scale, int B, int k0, int nk, float2* grids,
                          float2* partials, long long slots_per_b, int* counters, int nbins, int coils,
                          cudaStream_t st);
long long residual_loss_partials(int maxB, long long J);
cudaError_t launch_residual_loss(const float2* yhat, const float2* ymeas, const int* meas_idx, const float* dcf, int B,
                                 long long J, int nrows, float2* r2, double* partials, unsigned int* counter,
                                 float* loss, int* status, cudaStream_t st);

// Two-pass register FFT kernels (fft2.cu) for the specialised lengths; they
// return cudaErrorNotSupported for any other length (the Stockham kernels of
// fft.cu then run instead).
bool fft2_supported(int L);
cudaError_t launch_fft2_strided(const FftAxis& ax, int inverse, const float2* in, float2* out, int n_in,
                                int in_centred, int n_out, int out_centred, long long inner, long long outer,
                                cudaStream_t st);
cudaError_t launch_fft2_fwd_prologue(const Geo& g, const FftAxis& ax, const float2* x, const float2* S,
                                     const int* coil_idx, int B, int k0, int nk, const float* dinv1,
                                     const float* dinv2, const float* dinv3, float2* out, int* status,
                                     cudaStream_t st);
// Adjoint axis-3 FFT + epilogue with bulk-copy staged inputs (fft2_staged.cu).
bool fft2_epilogue_staged_ok(const Geo& g, const FftAxis& ax, const float2* in, const float2* S, int nk);
cudaError_t launch_fft2_epilogue_staged(const Geo& g, const FftAxis& ax, const float2* in, const float2* S,
                                        const int* coil_idx, int B, int k0, int nk, const float* dinv1,
                                        const float* dinv2, const float* dinv3, float2* out, int accumulate,
                                        int* status, cudaStream_t st);
// Forward prologue + axis-3 FFT with bulk-copy staged inputs (fft2_staged.cu).
bool fft2_prologue_staged_ok(const Geo& g, const FftAxis& ax, const float2* x, const float2* S, int nk);
cudaError_t launch_fft2_prologue_staged(const Geo& g, const FftAxis& ax, const float2* x, const float2* S,
                                        const int* coil_idx, int B, int k0, int nk, const float* dinv1,
                                        const float* dinv2, const float* dinv3, float2* out, int* status,
                                        cudaStream_t st);
cudaError_t launch_fft2_adj_epilogue(const Geo& g, const FftAxis& ax, const float2* in, const float2* S,
                                     const int* coil_idx, int B, int k0, int nk, const float* dinv1,
                                     const float* dinv2, const float* dinv3, float2* out, int accumulate,
                                     int* status, cudaStream_t st);

// Total variation of the image (tv.cu).
long long tv_partials(int K, int N1, int N2, int N3);

// Count kernel launches made outside the plan's run() wrapper (sdp_launch_count).
void note_launches(long long n);
cudaError_t launch_tv_value(const Geo& g, const float2* x, float eps, float lambda, double* partials,
                            unsigned int* counter, float* out, cudaStream_t st);
cudaError_t launch_tv_grad(const Geo& g, const float2* x, float eps, float lambda, const float* scale, float2* out,
                           int accumulate, cudaStream_t st);

// Host helpers.
bool fft_factor(int L, FftAxis* ax);
std::vector<float2> fft_twiddles(int L);

}  // namespace sdp
