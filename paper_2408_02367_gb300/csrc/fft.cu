// Mixed-radix (2, 3, 4, 5) 3D FFT passes over the oversampled grid, one axis
// per launch, with the lines of a CTA staged in shared memory.
//
// Steps A1/A2 (forward) and A6/A7 (adjoint) of the gridding NUFFT that
// evaluates the per-coil operator of StoDIP, Sec. 2 Eq. 1 / Sec. 2.1 Eq. 3:
//   forward  u = S_c x_k / psi_hat placed at n mod M, U = DFT_M(u) (sign -1)
//   adjoint  h = DFT_M^{-1}(H) unnormalised (sign +1), cropped at n mod M,
//            out_k += conj(S_c) h / psi_hat, summed over the coil minibatch.
// The paper names the NUFFT library it calls and gives no FFT design; this is a
// Stockham autosort FFT (Stockham 1966; GPU formulation of Govindaraju et al.
// 2008) run on NL columns at once so that shared-memory rows are read by
// consecutive lanes.
//
// Pruning: the forward input of every axis holds only N_d of the M_d points
// (zero padding), and the adjoint keeps only N_d outputs; the passes read and
// write just those rows, so the intermediate arrays are [..][N_d][..] wide.
#include <cmath>
#include <cstdlib>

#include "index_map.cuh"
#include "sdp_internal.cuh"

namespace sdp {
namespace {

constexpr int NL = 16;        // lines per CTA (shared-memory columns)
constexpr int NLP = NL + 1;   // padded row pitch in float2, avoids bank conflicts
constexpr int kThreads = 256;

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_j(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// Small DFTs V[q] = sum_r v[r] exp(-+2 pi i r q / R), in place.
template <int R, bool INV>
struct Dft;

template <bool INV>
struct Dft<2, INV> {
    __device__ __forceinline__ static void run(float2* v) {
        float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <bool INV>
struct Dft<3, INV> {
    __device__ __forceinline__ static void run(float2* v) {
        // cos(2 pi / 3) = -1/2, sin(2 pi / 3) = sqrt(3)/2
        const float s3 = 0.86602540378443864676f;
        float2 t = cadd(v[1], v[2]);
        float2 d = csub(v[1], v[2]);
        float2 m = make_float2(v[0].x - 0.5f * t.x, v[0].y - 0.5f * t.y);
        float2 jd = mul_j<INV>(cscale(d, s3));
        v[0] = cadd(v[0], t);
        v[1] = cadd(m, jd);
        v[2] = csub(m, jd);
    }
};

template <bool INV>
struct Dft<4, INV> {
    __device__ __forceinline__ static void run(float2* v) {
        float2 a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
        float2 a2 = cadd(v[1], v[3]), a3 = mul_j<INV>(csub(v[1], v[3]));
        v[0] = cadd(a0, a2);
        v[2] = csub(a0, a2);
        v[1] = cadd(a1, a3);
        v[3] = csub(a1, a3);
    }
};

template <bool INV>
struct Dft<5, INV> {
    __device__ __forceinline__ static void run(float2* v) {
        // cos(2 pi/5), cos(4 pi/5), sin(2 pi/5), sin(4 pi/5)
        const float c1 = 0.30901699437494742410f, c2 = -0.80901699437494742410f;
        const float s1 = 0.95105651629515357212f, s2 = 0.58778525229247312917f;
        float2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
        float2 d1 = csub(v[1], v[4]), d2 = csub(v[2], v[3]);
        float2 m1 = make_float2(v[0].x + c1 * t1.x + c2 * t2.x, v[0].y + c1 * t1.y + c2 * t2.y);
        float2 m2 = make_float2(v[0].x + c2 * t1.x + c1 * t2.x, v[0].y + c2 * t1.y + c1 * t2.y);
        float2 e1 = mul_j<INV>(make_float2(s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y));
        float2 e2 = mul_j<INV>(make_float2(s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y));
        v[0] = cadd(v[0], cadd(t1, t2));
        v[1] = cadd(m1, e1);
        v[4] = csub(m1, e1);
        v[2] = cadd(m2, e2);
        v[3] = csub(m2, e2);
    }
};

// One Stockham stage of radix R on the NL columns of src [L][NLP] -> dst.
template <int R, bool INV>
__device__ __forceinline__ void stockham_stage(const float2* __restrict__ src, float2* __restrict__ dst,
                                               const float2* __restrict__ tw, int L, int Ns) {
    const int nbf = L / R;
    const int tunit = L / (Ns * R);
    for (int e = threadIdx.x; e < nbf * NL; e += blockDim.x) {
        const int c = e % NL;
        const int j = e / NL;
        const int k = j % Ns;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[(j + r * nbf) * NLP + c];
        const int ts = k * tunit;
#pragma unroll
        for (int r = 1; r < R; ++r) {
            float2 w = tw[r * ts];
            if (INV) w.y = -w.y;
            v[r] = cmul(v[r], w);
        }
        Dft<R, INV>::run(v);
        const int base = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[(base + r * Ns) * NLP + c] = v[r];
    }
}

// Full FFT of the NL columns in `a` (scratch `b`); returns the buffer holding the result.
template <bool INV>
__device__ float2* fft_columns(float2* a, float2* b, const float2* tw, const FftAxis& ax) {
    int Ns = 1;
    for (int s = 0; s < ax.nst; ++s) {
        const int R = ax.radix[s];
        if (R == 4)
            stockham_stage<4, INV>(a, b, tw, ax.L, Ns);
        else if (R == 2)
            stockham_stage<2, INV>(a, b, tw, ax.L, Ns);
        else if (R == 5)
            stockham_stage<5, INV>(a, b, tw, ax.L, Ns);
        else
            stockham_stage<3, INV>(a, b, tw, ax.L, Ns);
        __syncthreads();
        float2* t = a;
        a = b;
        b = t;
        Ns *= R;
    }
    return a;
}

__device__ __forceinline__ int wrap_mod(int v, int L) {
    v %= L;
    return v < 0 ? v + L : v;
}

// Strided axis: lines of length n_in along a non-contiguous axis of
// in[outer][n_in][inner]; output out[outer][n_out][inner].  CTA = NL columns.
template <bool INV>
__global__ void __launch_bounds__(kThreads) fft_strided_kernel(const float2* __restrict__ in,
                                                              float2* __restrict__ out, FftAxis ax, int n_in,
                                                              int in_centred, int n_out, int out_centred,
                                                              long long inner, long long ncolblk) {
    extern __shared__ float2 smem[];
    const int L = ax.L;
    float2* tw = smem;
    float2* bufa = smem + L;
    float2* bufb = bufa + L * NLP;
    const long long blk = blockIdx.x;
    const long long o = blk / ncolblk;
    const long long c0 = (blk - o * ncolblk) * NL;
    const int ncols = (int)((inner - c0) < NL ? (inner - c0) : NL);
    for (int i = threadIdx.x; i < L; i += blockDim.x) tw[i] = ax.tw[i];
    const float2* src = in + o * (long long)n_in * inner + c0;
    const int h_in = in_centred ? n_in / 2 : 0;
    for (int e = threadIdx.x; e < L * NL; e += blockDim.x) {
        const int p = e / NL, c = e % NL;
        int r = p + h_in;
        if (r >= L) r -= L;
        float2 v = make_float2(0.f, 0.f);
        if (r < n_in && c < ncols) v = src[(long long)r * inner + c];
        bufa[p * NLP + c] = v;
    }
    __syncthreads();
    const float2* res = fft_columns<INV>(bufa, bufb, tw, ax);
    float2* dst = out + o * (long long)n_out * inner + c0;
    const int h_out = out_centred ? n_out / 2 : 0;
    for (int e = threadIdx.x; e < n_out * NL; e += blockDim.x) {
        const int r = e / NL, c = e % NL;
        const int p = out_centred ? wrap_mod(r - h_out, L) : r;
        if (c < ncols) dst[(long long)r * inner + c] = res[p * NLP + c];
    }
}

__device__ __forceinline__ void set_status(int* status, int code) {
    if (status) atomicCAS(status, 0, code);
}

// Forward A1 fused with the axis-3 FFT.  Lines l = row * nk + kk over
// row = i1 * N2 + i2; for each coil b of the batch the line is
// S_c[row][:] x_{k0+kk}[row][:] / psi_hat placed at (i3 - N3/2) mod M3.
// out[b][row][0..M3)[kk] (channel-interleaved; the store has the line index
// fastest so the channels of one grid point are written together).
__global__ void __launch_bounds__(kThreads) fwd_prologue_fft3_kernel(
    Geo g, FftAxis ax, const float2* __restrict__ x, const float2* __restrict__ S,
    const int* __restrict__ coil_idx, int B, int k0, int nk, const float* __restrict__ d1,
    const float* __restrict__ d2, const float* __restrict__ d3, float2* __restrict__ out, int* status) {
    extern __shared__ float2 smem[];
    const int L = ax.L;   // M3
    float2* tw = smem;
    float2* bufa = smem + L;
    float2* bufb = bufa + L * NLP;
    const int N2 = g.N[1], N3 = g.N[2];
    const long long nrows = (long long)g.N[0] * N2;
    const long long nlines = nrows * nk;
    const long long l0 = (long long)blockIdx.x * NL;
    const long long nvox = nrows * N3;
    for (int i = threadIdx.x; i < L; i += blockDim.x) tw[i] = ax.tw[i];
    const int h = N3 / 2;
    for (int b = 0; b < B; ++b) {
        int c = coil_idx[b];
        const bool cok = (c >= 0 && c < g.C);
        if (!cok && threadIdx.x == 0) set_status(status, SDP_ERR_BOUNDS);
        // load: e -> (line l, position p), p fastest so global reads are coalesced
        for (int e = threadIdx.x; e < NL * L; e += blockDim.x) {
            const int l = e / L, p = e - (e / L) * L;
            const long long gl = l0 + l;
            int i3 = p + h;
            if (i3 >= L) i3 -= L;
            float2 v = make_float2(0.f, 0.f);
            if (gl < nlines && i3 < N3 && cok) {
                const long long row = gl / nk;
                const int kk = (int)(gl - row * nk);
                const int i1 = (int)(row / N2), i2 = (int)(row - (long long)i1 * N2);
                const float2 xv = x[(long long)(k0 + kk) * nvox + row * N3 + i3];
                const float2 sv = S[(long long)c * nvox + row * N3 + i3];
                const float dd = d1[i1] * d2[i2] * d3[i3];
                v = cscale(cmul(sv, xv), dd);
            }
            bufa[p * NLP + l] = v;
        }
        __syncthreads();
        const float2* res = fft_columns<false>(bufa, bufb, tw, ax);
        for (int e = threadIdx.x; e < NL * L; e += blockDim.x) {
            const imap::LinePos lp = imap::stockham_elem(e, NL);
            const int p = lp.p, l = lp.l;
            const long long gl = l0 + l;
            if (gl < nlines) {
                const imap::LineRowChannel rc = imap::line_split(gl, nk);
                out[imap::line_elem((long long)b * nrows + rc.row, L, p, nk, rc.kk)] = res[p * NLP + l];
            }
        }
        __syncthreads();
    }
}

// Adjoint axis-3 inverse FFT fused with A7: for each coil b, invert the line
// (in[b][row][0..M3)[kk], channel-interleaved),
// keep the N3 centred outputs, multiply by conj(S_c), sum over b, divide by
// psi_hat and write (or add into) out[k0+kk][row][:].
__global__ void __launch_bounds__(kThreads) adj_fft3_epilogue_kernel(
    Geo g, FftAxis ax, const float2* __restrict__ in, const float2* __restrict__ S,
    const int* __restrict__ coil_idx, int B, int k0, int nk, const float* __restrict__ d1,
    const float* __restrict__ d2, const float* __restrict__ d3, float2* __restrict__ out, int accumulate,
    int* status) {
    extern __shared__ float2 smem[];
    const int L = ax.L;   // M3
    const int N2 = g.N[1], N3 = g.N[2];
    float2* tw = smem;
    float2* bufa = smem + L;
    float2* bufb = bufa + L * NLP;
    float2* acc = bufb + L * NLP;   // [N3][NLP]
    const long long nrows = (long long)g.N[0] * N2;
    const long long nlines = nrows * nk;
    const long long l0 = (long long)blockIdx.x * NL;
    const long long nvox = nrows * N3;
    for (int i = threadIdx.x; i < L; i += blockDim.x) tw[i] = ax.tw[i];
    for (int e = threadIdx.x; e < N3 * NLP; e += blockDim.x) acc[e] = make_float2(0.f, 0.f);
    const int h = N3 / 2;
    for (int b = 0; b < B; ++b) {
        int c = coil_idx[b];
        const bool cok = (c >= 0 && c < g.C);
        if (!cok && threadIdx.x == 0) set_status(status, SDP_ERR_BOUNDS);
        for (int e = threadIdx.x; e < NL * L; e += blockDim.x) {
            const imap::LinePos lp = imap::stockham_elem(e, NL);
            const int p = lp.p, l = lp.l;
            const long long gl = l0 + l;
            float2 v = make_float2(0.f, 0.f);
            if (gl < nlines) {
                const imap::LineRowChannel rc = imap::line_split(gl, nk);
                v = in[imap::line_elem((long long)b * nrows + rc.row, L, p, nk, rc.kk)];
            }
            bufa[p * NLP + l] = v;
        }
        __syncthreads();
        const float2* res = fft_columns<true>(bufa, bufb, tw, ax);
        if (cok) {
            for (int e = threadIdx.x; e < NL * N3; e += blockDim.x) {
                const int l = e / N3, o = e - (e / N3) * N3;
                const long long gl = l0 + l;
                if (gl < nlines) {
                    const long long row = gl / nk;
                    int p = o - h;
                    if (p < 0) p += L;
                    float2 s = S[(long long)c * nvox + row * N3 + o];
                    s.y = -s.y;
                    const float2 r = res[p * NLP + l];
                    float2 a = acc[o * NLP + l];
                    a = cadd(a, cmul(s, r));
                    acc[o * NLP + l] = a;
                }
            }
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < NL * N3; e += blockDim.x) {
        const int l = e / N3, o = e - (e / N3) * N3;
        const long long gl = l0 + l;
        if (gl < nlines) {
            const long long row = gl / nk;
            const int kk = (int)(gl - row * nk);
            const int i1 = (int)(row / N2), i2 = (int)(row - (long long)i1 * N2);
            const float dd = d1[i1] * d2[i2] * d3[o];
            float2 v = cscale(acc[o * NLP + l], dd);
            float2* dst = out + (long long)(k0 + kk) * nvox + row * N3 + o;
            if (accumulate) v = cadd(v, *dst);
            *dst = v;
        }
    }
}

size_t smem_fft_bytes(int L) { return (size_t)(L + 2 * L * NLP) * sizeof(float2); }

template <typename KernelT>
cudaError_t ensure_smem(KernelT kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// SDP_FFT_GENERIC=1 forces the Stockham kernels for every length (tests use it
// to compare the two FFT engines).
const bool g_generic_only = [] {
    const char* e = std::getenv("SDP_FFT_GENERIC");
    return e && e[0] == '1';
}();

}  // namespace

bool fft_factor(int L, FftAxis* ax) {
    ax->L = L;
    ax->nst = 0;
    int m = L;
    const int order[4] = {4, 2, 3, 5};
    for (int pi = 0; pi < 4; ++pi) {
        const int p = order[pi];
        while (m % p == 0) {
            if (ax->nst >= kMaxRadixStages) return false;
            ax->radix[ax->nst++] = p;
            m /= p;
        }
    }
    return m == 1 && L >= 2;
}

std::vector<float2> fft_twiddles(int L) {
    std::vector<float2> tw(L);
    for (int m = 0; m < L; ++m) {
        // exp(-2 pi i m / L) in float64, rounded once to float32
        const double a = -2.0 * M_PI * (double)m / (double)L;
        tw[m] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    return tw;
}

cudaError_t launch_fft_strided(const FftAxis& ax, int inverse, const float2* in, float2* out, int n_in,
                               int in_centred, int n_out, int out_centred, long long inner, long long outer,
                               cudaStream_t st) {
    if (fft2_supported(ax.L) && !g_generic_only && !ax.generic)
        return launch_fft2_strided(ax, inverse, in, out, n_in, in_centred, n_out, out_centred, inner, outer, st);
    const size_t sm = smem_fft_bytes(ax.L);
    const long long ncolblk = (inner + NL - 1) / NL;
    const long long nblk = ncolblk * outer;
    if (nblk <= 0) return cudaSuccess;
    if (nblk > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    cudaError_t e;
    if (inverse) {
        if ((e = ensure_smem(fft_strided_kernel<true>, sm)) != cudaSuccess) return e;
        fft_strided_kernel<true><<<(unsigned)nblk, kThreads, sm, st>>>(in, out, ax, n_in, in_centred, n_out,
                                                                      out_centred, inner, ncolblk);
    } else {
        if ((e = ensure_smem(fft_strided_kernel<false>, sm)) != cudaSuccess) return e;
        fft_strided_kernel<false><<<(unsigned)nblk, kThreads, sm, st>>>(in, out, ax, n_in, in_centred, n_out,
                                                                       out_centred, inner, ncolblk);
    }
    return cudaGetLastError();
}

cudaError_t launch_fwd_prologue_fft3(const Geo& g, const FftAxis& ax, const float2* x, const float2* S,
                                     const int* coil_idx, int B, int k0, int nk, const float* dinv1,
                                     const float* dinv2, const float* dinv3, float2* out, int* status,
                                     cudaStream_t st) {
    if (fft2_supported(ax.L) && !g_generic_only && !ax.generic) {
        if ((ax.staged & 1) && fft2_prologue_staged_ok(g, ax, x, S, nk))
            return launch_fft2_prologue_staged(g, ax, x, S, coil_idx, B, k0, nk, dinv1, dinv2, dinv3, out, status, st);
        return launch_fft2_fwd_prologue(g, ax, x, S, coil_idx, B, k0, nk, dinv1, dinv2, dinv3, out, status, st);
    }
    const size_t sm = smem_fft_bytes(ax.L);
    const long long nlines = (long long)g.N[0] * g.N[1] * nk;
    const long long nblk = (nlines + NL - 1) / NL;
    cudaError_t e;
    if ((e = ensure_smem(fwd_prologue_fft3_kernel, sm)) != cudaSuccess) return e;
    fwd_prologue_fft3_kernel<<<(unsigned)nblk, kThreads, sm, st>>>(g, ax, x, S, coil_idx, B, k0, nk, dinv1,
                                                                   dinv2, dinv3, out, status);
    return cudaGetLastError();
}

cudaError_t launch_adj_fft3_epilogue(const Geo& g, const FftAxis& ax, const float2* in, const float2* S,
                                     const int* coil_idx, int B, int k0, int nk, const float* dinv1,
                                     const float* dinv2, const float* dinv3, float2* out, int accumulate,
                                     int* status, cudaStream_t st) {
    if (fft2_supported(ax.L) && !g_generic_only && !ax.generic) {
        if ((ax.staged & 2) && fft2_epilogue_staged_ok(g, ax, in, S, nk))
            return launch_fft2_epilogue_staged(g, ax, in, S, coil_idx, B, k0, nk, dinv1, dinv2, dinv3, out,
                                               accumulate, status, st);
        return launch_fft2_adj_epilogue(g, ax, in, S, coil_idx, B, k0, nk, dinv1, dinv2, dinv3, out, accumulate,
                                        status, st);
    }
    const size_t sm = smem_fft_bytes(ax.L) + (size_t)g.N[2] * NLP * sizeof(float2);
    const long long nlines = (long long)g.N[0] * g.N[1] * nk;
    const long long nblk = (nlines + NL - 1) / NL;
    cudaError_t e;
    if ((e = ensure_smem(adj_fft3_epilogue_kernel, sm)) != cudaSuccess) return e;
    adj_fft3_epilogue_kernel<<<(unsigned)nblk, kThreads, sm, st>>>(g, ax, in, S, coil_idx, B, k0, nk, dinv1,
                                                                   dinv2, dinv3, out, accumulate, status);
    return cudaGetLastError();
}

}  // namespace sdp
