// Two-pass register FFT building blocks (included by fft2.cu and batch.cu):
// compile-time trigonometry, register DFTs, and the bodies of the strided pass,
// the fused forward prologue + axis-3 pass and the fused axis-3 pass + adjoint
// epilogue, each acting on one CTA-sized unit of work with the caller's shared
// memory.  fft2.cu wraps each body in a kernel over one plan; batch.cu calls
// them for the units of several plans in one launch.
//
// Two-pass register FFT along one axis of the oversampled grid (steps A2 / A6
// of the gridding NUFFT that evaluates StoDIP's per-coil operator, Sec. 2
// Eq. 1 and Sec. 2.1 Eq. 3), for lengths L = A * B with compile-time A and B.
//
// With n = B a + b and k = q1 + A q2 (a, q1 < A; b, q2 < B):
//   X[q1 + A q2] = sum_b w_B^{b q2} ( w_L^{b q1} sum_a x[B a + b] w_A^{a q1} )
// Pass 1: a thread holds the A points x[B a + b] of one (line, b) in
// registers, does the length-A DFT there, multiplies by w_L^{b q1} and writes
// the A results to shared memory.  Pass 2: a thread reads the B values of one
// (line, q1), does the length-B DFT in registers and writes X[q1 + A q2]
// straight to global memory.  So each point crosses shared memory once, and
// every index and every twiddle inside the small DFTs is a compile-time
// constant (cos / sin evaluated by constexpr series in float64, rounded once).
//
// The pruning of the zero-padded forward input (N of M rows) and of the
// cropped adjoint output is folded into the global loads / stores, and the
// fused forward prologue (S_c x_k / psi_hat) and adjoint epilogue
// (conj(S_c) h / psi_hat summed over the coil minibatch) act on the registers
// of pass 1 / pass 2.  Lengths without a specialisation fall back to the
// Stockham kernels of fft.cu.

#pragma once

#include <utility>

#include "index_map.cuh"
#include "sdp_internal.cuh"

namespace sdp {
namespace {


// ---------------- compile-time trigonometry ----------------
__host__ __device__ constexpr double cx_pi() { return 3.14159265358979323846264338327950288; }

__host__ __device__ constexpr double cx_sin_series(double x) {
    double term = x, sum = x;
    const double x2 = x * x;
    for (int n = 1; n < 14; ++n) {
        term *= -x2 / ((2.0 * n) * (2.0 * n + 1.0));
        sum += term;
    }
    return sum;
}

__host__ __device__ constexpr double cx_cos_series(double x) {
    double term = 1.0, sum = 1.0;
    const double x2 = x * x;
    for (int n = 1; n < 14; ++n) {
        term *= -x2 / ((2.0 * n - 1.0) * (2.0 * n));
        sum += term;
    }
    return sum;
}

// cos and sin of 2 pi e / N for integers: reduce to the nearest multiple of a
// quarter turn, |r| <= pi/4, then the series above.
__host__ __device__ constexpr double cx_cos2pi(int e, int N) {
    e %= N;
    if (e < 0) e += N;
    const int qq = (int)((8LL * e) / N + 1) / 2;      // nearest quarter turn, 0..4
    const double r = 2.0 * cx_pi() * (double)e / (double)N - qq * (cx_pi() / 2.0);
    switch (qq % 4) {
        case 0: return cx_cos_series(r);
        case 1: return -cx_sin_series(r);
        case 2: return -cx_cos_series(r);
        default: return cx_sin_series(r);
    }
}

__host__ __device__ constexpr double cx_sin2pi(int e, int N) {
    e %= N;
    if (e < 0) e += N;
    const int qq = (int)((8LL * e) / N + 1) / 2;
    const double r = 2.0 * cx_pi() * (double)e / (double)N - qq * (cx_pi() / 2.0);
    switch (qq % 4) {
        case 0: return cx_sin_series(r);
        case 1: return cx_cos_series(r);
        case 2: return -cx_sin_series(r);
        default: return -cx_cos_series(r);
    }
}

// exp(-2 pi i e / N) (forward) or exp(+2 pi i e / N) (inverse) as float constants.
template <int N, int E, bool INV>
struct TwC {
    static constexpr float c = (float)cx_cos2pi(E, N);
    static constexpr float s = (float)(INV ? cx_sin2pi(E, N) : -cx_sin2pi(E, N));
};

// ---------------- complex helpers ----------------
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
template <bool INV>
__device__ __forceinline__ float2 mul_j(float2 a) {   // * (-i) forward, * (+i) inverse
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <int I, int N>
struct StaticFor {
    template <class F>
    __device__ __forceinline__ static void run(F&& f) {
        f(std::integral_constant<int, I>{});
        StaticFor<I + 1, N>::run(f);
    }
};
template <int N>
struct StaticFor<N, N> {
    template <class F>
    __device__ __forceinline__ static void run(F&&) {}
};

// ---------------- register DFTs ----------------
__host__ __device__ constexpr int first_radix(int n) {
    return (n % 4 == 0 && n != 8) ? 4 : (n % 2 == 0 ? 2 : (n % 3 == 0 ? 3 : 5));
}

template <int N, bool INV>
struct RegDft;

template <bool INV>
struct RegDft<1, INV> {
    template <class T>
    __device__ __forceinline__ static void run(T&) {}
};

template <bool INV>
struct RegDft<2, INV> {
    template <class T>
    __device__ __forceinline__ static void run(T& v) {
        const float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <bool INV>
struct RegDft<3, INV> {
    template <class T>
    __device__ __forceinline__ static void run(T& v) {
        const float s3 = 0.86602540378443864676f;   // sin(2 pi / 3)
        const float2 t = cadd(v[1], v[2]);
        const float2 d = csub(v[1], v[2]);
        const float2 m = make_float2(v[0].x - 0.5f * t.x, v[0].y - 0.5f * t.y);
        const float2 jd = mul_j<INV>(cscale(d, s3));
        v[0] = cadd(v[0], t);
        v[1] = cadd(m, jd);
        v[2] = csub(m, jd);
    }
};

template <bool INV>
struct RegDft<4, INV> {
    template <class T>
    __device__ __forceinline__ static void run(T& v) {
        const float2 a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
        const float2 a2 = cadd(v[1], v[3]), a3 = mul_j<INV>(csub(v[1], v[3]));
        v[0] = cadd(a0, a2);
        v[2] = csub(a0, a2);
        v[1] = cadd(a1, a3);
        v[3] = csub(a1, a3);
    }
};

template <bool INV>
struct RegDft<5, INV> {
    template <class T>
    __device__ __forceinline__ static void run(T& v) {
        const float c1 = 0.30901699437494742410f, c2 = -0.80901699437494742410f;   // cos(2pi/5), cos(4pi/5)
        const float s1 = 0.95105651629515357212f, s2 = 0.58778525229247312917f;    // sin(2pi/5), sin(4pi/5)
        const float2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
        const float2 d1 = csub(v[1], v[4]), d2 = csub(v[2], v[3]);
        const float2 m1 = make_float2(v[0].x + c1 * t1.x + c2 * t2.x, v[0].y + c1 * t1.y + c2 * t2.y);
        const float2 m2 = make_float2(v[0].x + c2 * t1.x + c1 * t2.x, v[0].y + c2 * t1.y + c1 * t2.y);
        const float2 e1 = mul_j<INV>(make_float2(s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y));
        const float2 e2 = mul_j<INV>(make_float2(s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y));
        v[0] = cadd(v[0], cadd(t1, t2));
        v[1] = cadd(m1, e1);
        v[4] = csub(m1, e1);
        v[2] = cadd(m2, e2);
        v[3] = csub(m2, e2);
    }
};

// Generic N = R * M: DFT_R over x[m + M r] for each m, twiddle w_N^{m k1},
// then DFT_M over m for each k1, giving X[R k2 + k1].
template <int N, bool INV>
struct RegDft {
    template <class T>
    __device__ __forceinline__ static void run(T& v) {
        constexpr int R = first_radix(N);
        constexpr int M = N / R;
        float2 y[N];
        StaticFor<0, M>::run([&](auto mc) {
            constexpr int m = decltype(mc)::value;
            float2 t[R];
            StaticFor<0, R>::run([&](auto rc) {
                constexpr int r = decltype(rc)::value;
                t[r] = v[m + M * r];
            });
            RegDft<R, INV>::run(t);
            StaticFor<0, R>::run([&](auto kc) {
                constexpr int k1 = decltype(kc)::value;
                constexpr int e = (m * k1) % N;
                if constexpr (e == 0) {
                    y[m * R + k1] = t[k1];
                } else {
                    y[m * R + k1] = cmul(t[k1], make_float2(TwC<N, e, INV>::c, TwC<N, e, INV>::s));
                }
            });
        });
        StaticFor<0, R>::run([&](auto kc) {
            constexpr int k1 = decltype(kc)::value;
            float2 z[M];
            StaticFor<0, M>::run([&](auto mc) {
                constexpr int m = decltype(mc)::value;
                z[m] = y[m * R + k1];
            });
            RegDft<M, INV>::run(z);
            StaticFor<0, M>::run([&](auto kc2) {
                constexpr int k2 = decltype(kc2)::value;
                v[R * k2 + k1] = z[k2];
            });
        });
    }
};

__device__ __forceinline__ float2 twiddle(const float2* tw, int e, bool inv) {
    float2 w = tw[e];
    if (inv) w.y = -w.y;
    return w;
}

// ---------------- strided axis ----------------
// in[outer][n_in][inner] -> out[outer][n_out][inner], lines along the middle axis.
// One CTA-sized unit of work `blk` (column block x outer line); tw[L] and
// Y[L * NLT] are the caller's shared memory.
template <int A, int B, int NLT, bool INV>
__device__ __forceinline__ void fft2_strided_body(float2* tw, float2* Y, const float2* __restrict__ in,
                                                  float2* __restrict__ out, const float2* __restrict__ twg, int n_in,
                                                  int in_centred, int n_out, int out_centred, long long inner,
                                                  long long ncolblk, long long blk) {
    constexpr int L = A * B;
    const int tid = threadIdx.x;
    for (int i = tid; i < L; i += blockDim.x) tw[i] = twg[i];
    const long long o = blk / ncolblk;
    const long long c0 = (blk - o * ncolblk) * NLT;
    const int ncols = (int)((inner - c0) < NLT ? (inner - c0) : NLT);
    __syncthreads();
    if (tid < NLT * B) {
        const int c = tid % NLT, b = tid / NLT;
        const float2* src = in + o * (long long)n_in * inner + c0 + c;
        const int h = in_centred ? n_in / 2 : 0;
        float2 x[A];
        StaticFor<0, A>::run([&](auto ac) {
            constexpr int a = decltype(ac)::value;
            int r = B * a + b + h;       // source row of FFT position B a + b
            if (r >= L) r -= L;
            x[a] = (r < n_in && c < ncols) ? __ldg(src + (long long)r * inner) : make_float2(0.f, 0.f);
        });
        RegDft<A, INV>::run(x);
        StaticFor<0, A>::run([&](auto qc) {
            constexpr int q1 = decltype(qc)::value;
            const float2 v = q1 == 0 ? x[q1] : cmul(x[q1], twiddle(tw, b * q1, INV));
            Y[(q1 * B + b) * NLT + c] = v;
        });
    }
    __syncthreads();
    if (tid < NLT * A) {
        const int c = tid % NLT, q1 = tid / NLT;
        float2 z[B];
        StaticFor<0, B>::run([&](auto bc) {
            constexpr int b = decltype(bc)::value;
            z[b] = Y[(q1 * B + b) * NLT + c];
        });
        RegDft<B, INV>::run(z);
        float2* dst = out + o * (long long)n_out * inner + c0 + c;
        const int h = out_centred ? n_out / 2 : 0;
        StaticFor<0, B>::run([&](auto qc) {
            constexpr int q2 = decltype(qc)::value;
            int row = q1 + A * q2 + h;   // output row whose FFT index is q1 + A q2
            if (row >= L) row -= L;
            if (row < n_out && c < ncols) dst[(long long)row * inner] = z[q2];
        });
    }
}

// ---------------- forward prologue + axis 3 ----------------
// Lines l = row * nk + kk; block (line block, coil b) with the coil index the
// fastest, so the blocks of all coils of a line block run together and share
// the x lines in L2.  The line is S_c[row][:] x_{k0+kk}[row][:] / psi_hat
// placed at (i3 - N3/2) mod M3; it is written channel-interleaved,
// out[b][row][0..M3)[kk], with the lines the fastest thread index of pass 2
// so that a warp's stores of one grid point's channels are adjacent.
// One unit `blk` = (line block, coil): tw[L] and Y[NLT * (L + 1)] are the caller's shared memory.
template <int A, int B, int NLT>
__device__ __forceinline__ void fft2_prologue_body(
    float2* tw, float2* Y, const Geo& g, const float2* __restrict__ twg, const float2* __restrict__ x,
    const float2* __restrict__ S, const int* __restrict__ coil_idx, int Bc, int k0, int nk,
    const float* __restrict__ d1, const float* __restrict__ d2, const float* __restrict__ d3,
    float2* __restrict__ out, int* status, long long blk) {
    constexpr int L = A * B;
    constexpr int LP = L + 1;
    const int tid = threadIdx.x;
    for (int i = tid; i < L; i += blockDim.x) tw[i] = twg[i];
    const int N2 = g.N[1], N3 = g.N[2];
    const long long nrows = (long long)g.N[0] * N2;
    const long long nlines = nrows * nk;
    const long long nvox = nrows * N3;
    const unsigned ublk = (unsigned)blk;             // a grid's unit index fits 32 bits
    const int bb = (int)(ublk % (unsigned)Bc);
    const long long l0 = (long long)(ublk / (unsigned)Bc) * NLT;
    const int h = N3 / 2;
    const int c = coil_idx[bb];
    const bool cok = c >= 0 && c < g.C;
    if (!cok && tid == 0 && status) atomicCAS(status, 0, SDP_ERR_BOUNDS);
    __syncthreads();
    if (tid < NLT * B) {
        const imap::LinePos r1 = imap::pos_fastest(tid, B);
        const int b1 = r1.p, l1 = r1.l;
        const long long gl = l0 + l1;
        float2 u[A];
        if (gl < nlines && cok) {
            const imap::LineRowChannel rc = imap::line_split(gl, nk);
            const long long row = rc.row;
            const int kk = rc.kk;
            const int i1 = (int)(row / N2), i2 = (int)(row - (long long)i1 * N2);
            const float d12 = d1[i1] * d2[i2];
            const float2* xr = x + (long long)(k0 + kk) * nvox + row * N3;
            const float2* Sr = S + (long long)c * nvox + row * N3;
            StaticFor<0, A>::run([&](auto ac) {
                constexpr int a = decltype(ac)::value;
                int i3 = B * a + b1 + h;
                if (i3 >= L) i3 -= L;
                u[a] = i3 < N3 ? cscale(cmul(__ldg(Sr + i3), __ldg(xr + i3)), d12 * __ldg(d3 + i3))
                               : make_float2(0.f, 0.f);
            });
        } else {
            StaticFor<0, A>::run([&](auto ac) { u[decltype(ac)::value] = make_float2(0.f, 0.f); });
        }
        RegDft<A, false>::run(u);
        StaticFor<0, A>::run([&](auto qc) {
            constexpr int q1 = decltype(qc)::value;
            Y[l1 * LP + q1 * B + b1] = q1 == 0 ? u[q1] : cmul(u[q1], twiddle(tw, b1 * q1, false));
        });
    }
    __syncthreads();
    if (tid < NLT * A) {
        const imap::LinePos r2 = imap::line_fastest(tid, NLT);
        const int l2 = r2.l, q1 = r2.p;
        const long long gl = l0 + l2;
        if (gl < nlines) {
            const imap::LineRowChannel rc = imap::line_split(gl, nk);
            const long long row = rc.row;
            const int kk = rc.kk;
            float2 z[B];
            StaticFor<0, B>::run([&](auto bc) {
                constexpr int b = decltype(bc)::value;
                z[b] = Y[l2 * LP + q1 * B + b];
            });
            RegDft<B, false>::run(z);
            float2* dst = out + imap::line_elem((long long)bb * nrows + row, L, q1, nk, kk);
            const int sq = A * nk;   // outputs q1 + A q2 are A grid points apart
            StaticFor<0, B>::run([&](auto qc) {
                constexpr int q2 = decltype(qc)::value;
                dst[q2 * sq] = z[q2];
            });
        }
    }
}

// ---------------- adjoint axis 3 + epilogue ----------------
// For each coil of the batch: inverse DFT of the grid line (channel-interleaved,
// in[b][row][0..M3)[kk]; pass 1 has the lines as its fastest thread index so a
// warp's loads of one grid point's channels are adjacent), keep the N3 centred
// outputs, multiply by conj(S_c); sum over the batch in registers; divide by
// psi_hat and write (or add into) out[k0+kk][row][:].
// One unit `blk` = line block (all coils of the minibatch): tw[L] and Y[NLT * (L + 1)] are the
// caller's shared memory.
template <int A, int B, int NLT>
__device__ __forceinline__ void fft2_epilogue_body(
    float2* tw, float2* Y, const Geo& g, const float2* __restrict__ twg, const float2* __restrict__ in,
    const float2* __restrict__ S, const int* __restrict__ coil_idx, int Bc, int k0, int nk,
    const float* __restrict__ d1, const float* __restrict__ d2, const float* __restrict__ d3,
    float2* __restrict__ out, int accumulate, int* status, long long blk) {
    constexpr int L = A * B;
    constexpr int LP = L + 1;
    const int tid = threadIdx.x;
    for (int i = tid; i < L; i += blockDim.x) tw[i] = twg[i];
    const int N2 = g.N[1], N3 = g.N[2];
    const long long nrows = (long long)g.N[0] * N2;
    const long long nlines = nrows * nk;
    const long long nvox = nrows * N3;
    const long long l0 = blk * NLT;
    const int h = N3 / 2;
    const imap::LinePos r1 = imap::line_fastest(tid, NLT);
    const int l1 = r1.l, b1 = r1.p;
    const bool p1 = tid < NLT * B;
    const long long gl1 = l0 + l1;
    const bool line1 = p1 && gl1 < nlines;
    long long row1 = 0;
    int kk1 = 0;
    if (line1) {
        const imap::LineRowChannel rc = imap::line_split(gl1, nk);
        row1 = rc.row;
        kk1 = rc.kk;
    }
    const imap::LinePos r2 = imap::pos_fastest(tid, A);
    const int q12 = r2.p, l2 = r2.l;
    const bool p2 = tid < NLT * A;
    const long long gl2 = l0 + l2;
    const bool line2 = p2 && gl2 < nlines;
    long long row2 = 0;
    int kk2 = 0;
    // output voxel of FFT index q1 + A q2 (>= N3 when cropped away)
    auto ovox = [&](int q2) {
        int o = q12 + A * q2 + h;
        return o >= L ? o - L : o;
    };
    float2 acc[B];
    if (line2) {
        const imap::LineRowChannel rc = imap::line_split(gl2, nk);
        row2 = rc.row;
        kk2 = rc.kk;
    }
    StaticFor<0, B>::run([&](auto qc) { acc[decltype(qc)::value] = make_float2(0.f, 0.f); });
    __syncthreads();
    for (int bb = 0; bb < Bc; ++bb) {
        const int c = coil_idx[bb];
        const bool cok = c >= 0 && c < g.C;
        if (!cok && tid == 0 && status) atomicCAS(status, 0, SDP_ERR_BOUNDS);
        if (p1) {
            float2 u[A];
            const float2* src = in + imap::line_elem((long long)bb * nrows + row1, L, b1, nk, kk1);
            const int sa = B * nk;   // FFT positions B a + b1 are B grid points apart
            StaticFor<0, A>::run([&](auto ac) {
                constexpr int a = decltype(ac)::value;
                u[a] = line1 ? __ldg(src) : make_float2(0.f, 0.f);
                src += sa;
            });
            RegDft<A, true>::run(u);
            StaticFor<0, A>::run([&](auto qc) {
                constexpr int q1 = decltype(qc)::value;
                Y[l1 * LP + q1 * B + b1] = q1 == 0 ? u[q1] : cmul(u[q1], twiddle(tw, b1 * q1, true));
            });
        }
        __syncthreads();
        if (line2 && cok) {
            float2 z[B];
            StaticFor<0, B>::run([&](auto bc) {
                constexpr int b = decltype(bc)::value;
                z[b] = Y[l2 * LP + q12 * B + b];
            });
            RegDft<B, true>::run(z);
            const float2* Sr = S + (long long)c * nvox + row2 * N3;
            StaticFor<0, B>::run([&](auto qc) {
                constexpr int q2 = decltype(qc)::value;
                const int o = ovox(q2);
                if (o < N3) {
                    float2 s = __ldg(Sr + o);
                    s.y = -s.y;
                    acc[q2] = cadd(acc[q2], cmul(s, z[q2]));
                }
            });
        }
        __syncthreads();
    }
    if (line2) {
        const int i1 = (int)(row2 / N2), i2 = (int)(row2 - (long long)i1 * N2);
        const float d12 = d1[i1] * d2[i2];
        float2* dst = out + (long long)(k0 + kk2) * nvox + row2 * N3;
        StaticFor<0, B>::run([&](auto qc) {
            constexpr int q2 = decltype(qc)::value;
            const int o = ovox(q2);
            if (o < N3) {
                float2 v = cscale(acc[q2], d12 * __ldg(d3 + o));
                if (accumulate) v = cadd(v, dst[o]);
                dst[o] = v;
            }
        });
    }
}

// ---------------- dispatch ----------------
// Lines per CTA: 16, or 8 for the long axes so the registers of a length-25 DFT fit.
template <int A, int B, int NLT = (A * B >= 240 ? 8 : 16)>
struct Shape {
    static constexpr int a = A, b = B, nl = NLT, threads = NLT * (A > B ? A : B);
};

template <class F>
bool with_shape(int L, F&& f) {
    switch (L) {
        case 48: f(Shape<8, 6>{}); return true;
        case 64: f(Shape<8, 8>{}); return true;
        case 80: f(Shape<10, 8>{}); return true;
        case 96: f(Shape<12, 8>{}); return true;
        case 100: f(Shape<10, 10>{}); return true;
        case 120: f(Shape<12, 10>{}); return true;
        case 128: f(Shape<16, 8>{}); return true;
        case 160: f(Shape<16, 10>{}); return true;
        case 200: f(Shape<20, 10>{}); return true;
        case 240: f(Shape<16, 15>{}); return true;
        case 250: f(Shape<25, 10>{}); return true;
        case 256: f(Shape<16, 16>{}); return true;
        default: return false;
    }
}

// The same shapes with 8 lines per CTA (a plan's tuning, for the fused axis-3 kernels).
template <class F>
bool with_shape8(int L, F&& f) {
    switch (L) {
        case 48: f(Shape<8, 6, 8>{}); return true;
        case 64: f(Shape<8, 8, 8>{}); return true;
        case 80: f(Shape<10, 8, 8>{}); return true;
        case 96: f(Shape<12, 8, 8>{}); return true;
        case 100: f(Shape<10, 10, 8>{}); return true;
        case 120: f(Shape<12, 10, 8>{}); return true;
        case 128: f(Shape<16, 8, 8>{}); return true;
        case 160: f(Shape<16, 10, 8>{}); return true;
        case 200: f(Shape<20, 10, 8>{}); return true;
        case 240: f(Shape<16, 15, 8>{}); return true;
        case 250: f(Shape<25, 10, 8>{}); return true;
        case 256: f(Shape<16, 16, 8>{}); return true;
        default: return false;
    }
}

// ... and with 4 lines per CTA.
template <class F>
bool with_shape4(int L, F&& f) {
    switch (L) {
        case 48: f(Shape<8, 6, 4>{}); return true;
        case 64: f(Shape<8, 8, 4>{}); return true;
        case 80: f(Shape<10, 8, 4>{}); return true;
        case 96: f(Shape<12, 8, 4>{}); return true;
        case 100: f(Shape<10, 10, 4>{}); return true;
        case 120: f(Shape<12, 10, 4>{}); return true;
        case 128: f(Shape<16, 8, 4>{}); return true;
        case 160: f(Shape<16, 10, 4>{}); return true;
        case 200: f(Shape<20, 10, 4>{}); return true;
        case 240: f(Shape<16, 15, 4>{}); return true;
        case 250: f(Shape<25, 10, 4>{}); return true;
        case 256: f(Shape<16, 16, 4>{}); return true;
        default: return false;
    }
}

// 32 columns per CTA for the strided passes (a plan's tuning); the shared staging
// of L x 32 complex values stays within the 48 KB of static shared memory up to L = 160.
template <class F>
bool with_shape32(int L, F&& f) {
    switch (L) {
        case 48: f(Shape<8, 6, 32>{}); return true;
        case 64: f(Shape<8, 8, 32>{}); return true;
        case 80: f(Shape<10, 8, 32>{}); return true;
        case 96: f(Shape<12, 8, 32>{}); return true;
        case 100: f(Shape<10, 10, 32>{}); return true;
        case 120: f(Shape<12, 10, 32>{}); return true;
        case 128: f(Shape<16, 8, 32>{}); return true;
        case 160: f(Shape<16, 10, 32>{}); return true;
        default: return false;
    }
}


// 16 columns per CTA for every length: the default of the strided passes.  (The fused
// axis-3 kernels keep 8 lines for lengths >= 240, where a length-25 DFT and the
// epilogue's coil sum need the registers; a strided pass holds one line's DFT only,
// and 16 columns make each row segment it reads or writes 128 contiguous bytes.)
template <class F>
bool with_shape16(int L, F&& f) {
    switch (L) {
        case 48: f(Shape<8, 6, 16>{}); return true;
        case 64: f(Shape<8, 8, 16>{}); return true;
        case 80: f(Shape<10, 8, 16>{}); return true;
        case 96: f(Shape<12, 8, 16>{}); return true;
        case 100: f(Shape<10, 10, 16>{}); return true;
        case 120: f(Shape<12, 10, 16>{}); return true;
        case 128: f(Shape<16, 8, 16>{}); return true;
        case 160: f(Shape<16, 10, 16>{}); return true;
        case 200: f(Shape<20, 10, 16>{}); return true;
        case 240: f(Shape<16, 15, 16>{}); return true;
        case 250: f(Shape<25, 10, 16>{}); return true;
        case 256: f(Shape<16, 16, 16>{}); return true;
        default: return false;
    }
}

// Strided passes: the column count of the plan's tuning where a kernel exists, else 16.
template <class F>
bool with_shape_cols(const FftAxis& ax, F&& f) {
    if (ax.cols == 32 && with_shape32(ax.L, f)) return true;
    if (ax.cols == 8) return with_shape8(ax.L, f);
    return with_shape16(ax.L, f);
}

template <class F>
bool with_shape_of(const FftAxis& ax, F&& f) {
    if (ax.lines == 4) return with_shape4(ax.L, f);
    return ax.lines == 8 ? with_shape8(ax.L, f) : with_shape(ax.L, f);
}

}  // namespace
}  // namespace sdp
