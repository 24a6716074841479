// Descriptors of a batched launch over several plans (batch.cu), filled by the
// C ABI (api.cu).  Not part of the public interface.
#pragma once

#include "sdp_internal.cuh"

namespace sdp {

constexpr int kMaxMvItems = 16;   // items per launch

// One strided FFT pass of an item: in[outer][n_in][inner] -> out[outer][n_out][inner].
struct MvPass {
    const float2* in;
    float2* out;
    int n_in, in_centred, n_out, out_centred;
    long long inner;
};

// One item of a batched call: its plan's geometry and tables, the call's
// pointers, and the item's slice of the plan's workspace.
struct MvItem {
    Geo g;
    int L[3];                 // grid lengths M1, M2, M3
    const float2* tw[3];      // twiddles of each axis
    const float* d[3];        // 1 / deapodisation per axis
    float2* x;                // forward: the TSMI read; adjoint: the TSMI written
    const float2* S;
    const int* coil_idx;
    int B;
    int accumulate;           // adjoint: add into x
    int* status;
    float2* bufA;             // workspace slices of this item's coils
    float2* bufB;
    MvPass pass[2];           // [0]: axis 1, [1]: axis 2
    const float4* pts;
    const int* tframe;
    const float* wts;
    const float2* V;
    float2* y;                // forward: written; adjoint: read through sa.y
    SpreadArgs sa;
    int nsub;
    int spread_pairs;         // 1: one spread warp holds two coils
    int interp_coils;         // coils per interpolation sweep over the samples (B: all at once)
    const int4* itiles;       // tiled interpolation: the plan's work items, their count, tiles per axis 2, 3
    int n_itiles;
    int nt2, nt3;
};

struct MvArgs {
    MvItem it[kMaxMvItems];
};

// Units of work of one launch: item i owns units [start[i], start[i + 1]).
struct MvUnits {
    int n;
    long long start[kMaxMvItems + 1];
};

bool mv_length_supported(int L);
bool mv_width_supported(int W);        // interpolation and spread kernels of the batched path
long long mv_fused_lines(int L);     // lines per CTA of the fused axis-3 kernels for length L
long long mv_strided_cols(int L);    // columns per CTA of the strided passes for length L
cudaError_t launch_mv_prologue(const MvArgs& a, const MvUnits& u, cudaStream_t st);
cudaError_t launch_mv_strided(const MvArgs& a, const MvUnits& u, int axis, int inverse, cudaStream_t st);
cudaError_t launch_mv_epilogue(const MvArgs& a, const MvUnits& u, cudaStream_t st);
cudaError_t launch_mv_interp(const MvArgs& a, const MvUnits& u, int W, int threads, cudaStream_t st);
// Tiled interpolation of several plans (interp_tiles.cu); u.start: prefix sums of work items.
cudaError_t launch_mv_interp_tiles(const MvArgs& a, const MvUnits& u, int W, int K, cudaStream_t st);
cudaError_t launch_mv_spread(const MvArgs& a, const MvUnits& u, int bin_width, int bin_depth, int W, int K,
                             cudaStream_t st);

}  // namespace sdp
