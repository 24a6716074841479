// Two-pass register FFT kernels over one plan (steps A2 / A6 of the gridding
// NUFFT that evaluates StoDIP's per-coil operator, Sec. 2 Eq. 1 and Sec. 2.1
// Eq. 3): each kernel is one CTA per unit of work of the body in
// fft2_impl.cuh, with static shared memory sized for its shape.
#include "fft2_impl.cuh"

namespace sdp {
namespace {

template <int A, int B, int NLT, bool INV>
__global__ void __launch_bounds__(NLT*(A > B ? A : B)) fft2_strided_kernel(const float2* __restrict__ in,
                                                                         float2* __restrict__ out,
                                                                         const float2* __restrict__ twg, int n_in,
                                                                         int in_centred, int n_out, int out_centred,
                                                                         long long inner, long long ncolblk) {
    __shared__ float2 tw[A * B];
    __shared__ float2 Y[A * B * NLT];
    fft2_strided_body<A, B, NLT, INV>(tw, Y, in, out, twg, n_in, in_centred, n_out, out_centred, inner, ncolblk,
                                      (long long)blockIdx.x);
}

template <int A, int B, int NLT>
__global__ void __launch_bounds__(NLT*(A > B ? A : B)) fft2_fwd_prologue_kernel(
    Geo g, const float2* __restrict__ twg, const float2* __restrict__ x, const float2* __restrict__ S,
    const int* __restrict__ coil_idx, int Bc, int k0, int nk, const float* __restrict__ d1,
    const float* __restrict__ d2, const float* __restrict__ d3, float2* __restrict__ out, int* status) {
    __shared__ float2 tw[A * B];
    __shared__ float2 Y[NLT * (A * B + 1)];
    fft2_prologue_body<A, B, NLT>(tw, Y, g, twg, x, S, coil_idx, Bc, k0, nk, d1, d2, d3, out, status,
                                  (long long)blockIdx.x);
}

template <int A, int B, int NLT>
__global__ void __launch_bounds__(NLT*(A > B ? A : B)) fft2_adj_epilogue_kernel(
    Geo g, const float2* __restrict__ twg, const float2* __restrict__ in, const float2* __restrict__ S,
    const int* __restrict__ coil_idx, int Bc, int k0, int nk, const float* __restrict__ d1,
    const float* __restrict__ d2, const float* __restrict__ d3, float2* __restrict__ out, int accumulate,
    int* status) {
    __shared__ float2 tw[A * B];
    __shared__ float2 Y[NLT * (A * B + 1)];
    fft2_epilogue_body<A, B, NLT>(tw, Y, g, twg, in, S, coil_idx, Bc, k0, nk, d1, d2, d3, out, accumulate, status,
                                  (long long)blockIdx.x);
}

}  // namespace

bool fft2_supported(int L) {
    return with_shape(L, [](auto) {});
}

cudaError_t launch_fft2_strided(const FftAxis& ax, int inverse, const float2* in, float2* out, int n_in,
                                int in_centred, int n_out, int out_centred, long long inner, long long outer,
                                cudaStream_t st) {
    cudaError_t err = cudaErrorNotSupported;
    with_shape_cols(ax, [&](auto sh) {
        using S = decltype(sh);
        const long long ncolblk = (inner + S::nl - 1) / S::nl;
        const long long nblk = ncolblk * outer;
        if (nblk <= 0) {
            err = cudaSuccess;
            return;
        }
        if (nblk > 0x7fffffffLL) {
            err = cudaErrorInvalidConfiguration;
            return;
        }
        if (inverse)
            fft2_strided_kernel<S::a, S::b, S::nl, true><<<(unsigned)nblk, S::threads, 0, st>>>(
                in, out, ax.tw, n_in, in_centred, n_out, out_centred, inner, ncolblk);
        else
            fft2_strided_kernel<S::a, S::b, S::nl, false><<<(unsigned)nblk, S::threads, 0, st>>>(
                in, out, ax.tw, n_in, in_centred, n_out, out_centred, inner, ncolblk);
        err = cudaGetLastError();
    });
    return err;
}

cudaError_t launch_fft2_fwd_prologue(const Geo& g, const FftAxis& ax, const float2* x, const float2* S,
                                     const int* coil_idx, int B, int k0, int nk, const float* dinv1,
                                     const float* dinv2, const float* dinv3, float2* out, int* status,
                                     cudaStream_t st) {
    const long long nlines = (long long)g.N[0] * g.N[1] * nk;
    cudaError_t err = cudaErrorNotSupported;
    with_shape_of(ax, [&](auto sh) {
        using Sh = decltype(sh);
        const long long nblk = (nlines + Sh::nl - 1) / Sh::nl * B;
        if (nblk > 0x7fffffffLL) {
            err = cudaErrorInvalidConfiguration;
            return;
        }
        fft2_fwd_prologue_kernel<Sh::a, Sh::b, Sh::nl><<<(unsigned)nblk, Sh::threads, 0, st>>>(
            g, ax.tw, x, S, coil_idx, B, k0, nk, dinv1, dinv2, dinv3, out, status);
        err = cudaGetLastError();
    });
    return err;
}

cudaError_t launch_fft2_adj_epilogue(const Geo& g, const FftAxis& ax, const float2* in, const float2* S,
                                     const int* coil_idx, int B, int k0, int nk, const float* dinv1,
                                     const float* dinv2, const float* dinv3, float2* out, int accumulate,
                                     int* status, cudaStream_t st) {
    const long long nlines = (long long)g.N[0] * g.N[1] * nk;
    cudaError_t err = cudaErrorNotSupported;
    with_shape_of(ax, [&](auto sh) {
        using Sh = decltype(sh);
        const long long nblk = (nlines + Sh::nl - 1) / Sh::nl;
        fft2_adj_epilogue_kernel<Sh::a, Sh::b, Sh::nl><<<(unsigned)nblk, Sh::threads, 0, st>>>(
            g, ax.tw, in, S, coil_idx, B, k0, nk, dinv1, dinv2, dinv3, out, accumulate, status);
        err = cudaGetLastError();
    });
    return err;
}

}  // namespace sdp
