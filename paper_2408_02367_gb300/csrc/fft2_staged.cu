// Forward prologue + axis-3 FFT (steps A1 and the first pass of A2 of the
// gridding NUFFT of StoDIP's per-coil operator, Sec. 2 Eq. 1, Sec. 2.1 Eq. 3)
// with its inputs staged by bulk copies; the adjoint's axis-3 FFT + epilogue
// (A6, A7) in the same form further down.
//
// The same arithmetic as fft2_prologue_body (fft2_impl.cuh), organised for
// the memory system: a unit of work is R whole image rows of one coil and all
// nk channels of the call (NL = R nk grid lines), and its inputs are whole
// contiguous runs of memory: S_c[row0 .. row0 + R)[:] and, per channel,
// x_k[row0 .. row0 + R)[:], R N3 complex values each.  One thread copies them
// into shared memory with cp.async.bulk (the TMA engine) completing on an
// mbarrier, so no register holds a load in flight.  CTAs are persistent and
// double-buffered: while a CTA transforms one unit, the copies of its next
// unit are already in flight.
//
// Pass 1 (thread = (line, b), b fastest): S x / psi_hat at the FFT positions
// B a + b of the line, read from shared memory, the length-A DFT in registers,
// the twiddles, into Y.  Pass 2 (thread = (row, q1, channel), channel
// fastest): the length-B DFT and the store of outputs q1 + A q2; for a fixed
// q2 the lanes of a warp write consecutive grid points' channels, one
// contiguous run of the channel-interleaved grid [b][row][m][kk].
//
// Every mbarrier wait is bounded (tma.cuh); after a wait that gives up, the
// CTA records SDP_ERR_TIMEOUT, waits (bounded) for the copies it still has in
// flight and returns.
#include <algorithm>

#include "fft2_impl.cuh"
#include "tma.cuh"

namespace sdp {
namespace {

// Threads per CTA: 512 for lengths of 200 and more (their units then hold twice the
// rows, halving the barriers per line; one CTA per SM), 256 below (three per SM).
template <int A, int B>
__host__ __device__ constexpr int staged_threads() { return A * B >= 200 ? 512 : 256; }

template <int A, int B>
__host__ __device__ constexpr int staged_lines() { return staged_threads<A, B>() / (A > B ? A : B); }

// Rows per unit for nk channels (0 when even one row's channels do not fit).
template <int A, int B>
__host__ __device__ constexpr int staged_rows(int nk) { return staged_lines<A, B>() / nk; }

// Dynamic shared memory: two mbarriers, the twiddles, Y, and two staging buffers
// of (1 + nk) R N3 complex values each.
template <int A, int B>
size_t staged_smem(int nk, int N3) {
    constexpr int L = A * B, LP = L + 1;
    const int R = staged_rows<A, B>(nk);
    const size_t head = 16 + (size_t)L * 8 + (size_t)R * nk * LP * 8;
    const size_t head16 = (head + 15) & ~(size_t)15;
    return head16 + 2 * (size_t)(1 + nk) * R * N3 * 8;
}

template <int A, int B>
__global__ void __launch_bounds__(staged_threads<A, B>(), (A * B >= 200 ? 1 : 3)) fft2_prologue_staged_kernel(
    Geo g, const float2* __restrict__ twg, const float2* __restrict__ x, const float2* __restrict__ S,
    const int* __restrict__ coil_idx, int Bc, int k0, int nk, const float* __restrict__ d1,
    const float* __restrict__ d2, const float* __restrict__ d3, float2* __restrict__ out, int* status) {
    constexpr int L = A * B;
    constexpr int LP = L + 1;
    extern __shared__ __align__(16) unsigned char smem[];
    const int R = staged_rows<A, B>(nk);
    const int NL = R * nk;
    const int N2 = g.N[1], N3 = g.N[2];
    const long long nrows = (long long)g.N[0] * N2;
    const long long nvox = nrows * N3;
    const int h = N3 / 2;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);                 // [2]
    float2* tw = reinterpret_cast<float2*>(smem + 16);                  // [L]
    float2* Y = tw + L;                                                  // [NL][LP]
    const size_t head = 16 + (size_t)L * 8 + (size_t)NL * LP * 8;
    float2* buf0 = reinterpret_cast<float2*>(smem + ((head + 15) & ~(size_t)15));
    const size_t bufn = (size_t)(1 + nk) * R * N3;                      // complex values per buffer
    const int tid = threadIdx.x;
    const long long nblk = (nrows + R - 1) / R;
    const long long nunits = nblk * Bc;

    for (int i = tid; i < L; i += blockDim.x) tw[i] = twg[i];
    if (tid == 0) {
        tma::mbar_init(bar, 1);
        tma::mbar_init(bar + 1, 1);
        tma::fence_init();
    }
    __syncthreads();

    // thread 0: copies of one unit into buffer s (S rows first, then the nk channels' rows)
    auto issue = [&](long long unit, int s) {
        const int bb = (int)(unit % Bc);
        const long long row0 = (unit / Bc) * R;
        const int nr = (int)(nrows - row0 < R ? nrows - row0 : R);
        const int c = coil_idx[bb];
        const bool cok = c >= 0 && c < g.C;
        const uint32_t run = (uint32_t)nr * N3 * 8;
        float2* bs = buf0 + s * bufn;
        tma::mbar_expect_tx(bar + s, run * (uint32_t)(nk + (cok ? 1 : 0)));
        if (cok) tma::bulk_g2s(bs, S + (long long)c * nvox + row0 * N3, run, bar + s);
        for (int kk = 0; kk < nk; ++kk)
            tma::bulk_g2s(bs + (size_t)(1 + kk) * R * N3, x + (long long)(k0 + kk) * nvox + row0 * N3, run, bar + s);
    };

    long long unit = blockIdx.x;
    if (tid == 0 && unit < nunits) issue(unit, 0);
    bool pending[2] = {unit < nunits, false};     // meaningful in thread 0
    for (int k = 0; unit < nunits; ++k) {
        const int s = k & 1;
        const long long next = unit + gridDim.x;
        if (tid == 0 && next < nunits) {
            issue(next, s ^ 1);
            pending[s ^ 1] = true;
        }
        const bool ok = tma::mbar_wait(bar + s, (uint32_t)(k >> 1) & 1u, status);
        if (tid == 0) pending[s] = !ok;
        if (!__syncthreads_and(ok)) {
            // a copy did not land within the limit: let the ones still in flight finish
            // (bounded) before the shared memory goes away
            if (tid == 0)
                for (int q = 0; q < 2; ++q)
                    if (pending[q]) tma::mbar_wait(bar + q, (uint32_t)((k + (q != s)) >> 1) & 1u, status);
            __syncthreads();
            return;
        }
        const int bb = (int)(unit % Bc);
        const long long row0 = (unit / Bc) * R;
        const int nr = (int)(nrows - row0 < R ? nrows - row0 : R);
        const int c = coil_idx[bb];
        const bool cok = c >= 0 && c < g.C;
        if (!cok && tid == 0 && status) atomicCAS(status, 0, SDP_ERR_BOUNDS);
        const float2* Ss = buf0 + s * bufn;
        if (tid < NL * B) {
            const imap::StagedLoad sl = imap::staged_load_role(tid, B, nk);
            const int l1 = sl.l, rr = sl.rr, kk = sl.kk, b1 = sl.b;
            float2 u[A];
            if (rr < nr && cok) {
                const long long row = row0 + rr;
                const int i1 = (int)(row / N2), i2 = (int)(row - (long long)i1 * N2);
                const float d12 = d1[i1] * d2[i2];
                const float2* Sr = Ss + rr * N3;
                const float2* xr = Ss + (size_t)(1 + kk) * R * N3 + rr * N3;
                StaticFor<0, A>::run([&](auto ac) {
                    constexpr int a = decltype(ac)::value;
                    int i3 = B * a + b1 + h;
                    if (i3 >= L) i3 -= L;
                    u[a] = i3 < N3 ? cscale(cmul(Sr[i3], xr[i3]), d12 * __ldg(d3 + i3)) : make_float2(0.f, 0.f);
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
        if (tid < NL * A) {
            const imap::StagedStore ss = imap::staged_store_role(tid, A, nk);
            const int kk = ss.kk, q1 = ss.q1, rr = ss.rr;
            if (rr < nr) {
                float2 z[B];
                const int l2 = rr * nk + kk;
                StaticFor<0, B>::run([&](auto bc) {
                    constexpr int b = decltype(bc)::value;
                    z[b] = Y[l2 * LP + q1 * B + b];
                });
                RegDft<B, false>::run(z);
                float2* dst = out + imap::line_elem((long long)bb * nrows + row0 + rr, L, q1, nk, kk);
                const int sq = A * nk;   // outputs q1 + A q2 are A grid points apart
                StaticFor<0, B>::run([&](auto qc) {
                    constexpr int q2 = decltype(qc)::value;
                    dst[q2 * sq] = z[q2];
                });
            }
        }
        __syncthreads();
        unit = next;
    }
}

// Adjoint axis-3 FFT + epilogue (the last pass of A6 and step A7) with its inputs
// staged by bulk copies: the same arithmetic as fft2_epilogue_body.  A unit is R
// whole rows (NL = R nk grid lines) and a step is (unit, coil): the coil's grid
// lines of the unit, in[b][row0 .. row0 + R)[0 .. L)[kk] (one contiguous run of
// R L nk values), and its coil-map rows S_c[row0 .. row0 + R)[:] (R N3 values),
// copied into shared memory by one thread with cp.async.bulk on an mbarrier.
// The steps are double-buffered like the prologue's units.  Pass 1 (thread =
// (line, b), line fastest): the length-A inverse DFT of the line's positions
// B a + b, the twiddles, into Y.  Pass 2 (thread = (line, q1), q1 fastest): the
// length-B inverse DFT, the crop to N3, conj(S_c) from shared memory, summed over
// the coils in registers; after a unit's last coil the thread scales by 1/psi_hat
// and stores, consecutive threads writing consecutive voxels of an image row.
template <int A, int B>
size_t staged_epi_smem(int nk, int N3) {
    constexpr int L = A * B, LP = L + 1;
    const int R = staged_rows<A, B>(nk);
    const size_t head = 16 + (size_t)L * 8 + (size_t)R * nk * LP * 8;
    const size_t head16 = (head + 15) & ~(size_t)15;
    return head16 + 2 * ((size_t)R * L * nk + (size_t)R * N3) * 8;
}

template <int A, int B>
__global__ void __launch_bounds__(staged_threads<A, B>(), (A * B >= 200 ? 1 : 3)) fft2_epilogue_staged_kernel(
    Geo g, const float2* __restrict__ twg, const float2* __restrict__ in, const float2* __restrict__ S,
    const int* __restrict__ coil_idx, int Bc, int k0, int nk, const float* __restrict__ d1,
    const float* __restrict__ d2, const float* __restrict__ d3, float2* __restrict__ out, int accumulate,
    int* status) {
    constexpr int L = A * B;
    constexpr int LP = L + 1;
    extern __shared__ __align__(16) unsigned char smem[];
    const int R = staged_rows<A, B>(nk);
    const int NL = R * nk;
    const int N2 = g.N[1], N3 = g.N[2];
    const long long nrows = (long long)g.N[0] * N2;
    const long long nvox = nrows * N3;
    const int h = N3 / 2;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);                 // [2]
    float2* tw = reinterpret_cast<float2*>(smem + 16);                  // [L]
    float2* Y = tw + L;                                                  // [NL][LP]
    const size_t head = 16 + (size_t)L * 8 + (size_t)NL * LP * 8;
    float2* buf0 = reinterpret_cast<float2*>(smem + ((head + 15) & ~(size_t)15));
    const size_t gridn = (size_t)R * L * nk;                            // grid lines, then coil-map rows
    const size_t bufn = gridn + (size_t)R * N3;
    const int tid = threadIdx.x;
    const long long nblk = (nrows + R - 1) / R;
    const long long myunits = (long long)blockIdx.x < nblk ? (nblk - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const long long nsteps = myunits * Bc;   // step k: unit blockIdx.x + (k / Bc) gridDim.x, coil k % Bc

    for (int i = tid; i < L; i += blockDim.x) tw[i] = twg[i];
    if (tid == 0) {
        tma::mbar_init(bar, 1);
        tma::mbar_init(bar + 1, 1);
        tma::fence_init();
    }
    __syncthreads();

    // thread 0: copies of step k into buffer s (the grid lines, then the coil map's rows)
    auto issue = [&](long long k, int s) {
        const long long row0 = ((long long)blockIdx.x + (k / Bc) * gridDim.x) * R;
        const int bb = (int)(k % Bc);
        const int nr = (int)(nrows - row0 < R ? nrows - row0 : R);
        const int c = coil_idx[bb];
        const bool cok = c >= 0 && c < g.C;
        const uint32_t gbytes = (uint32_t)nr * L * nk * 8, sbytes = (uint32_t)nr * N3 * 8;
        float2* bs = buf0 + s * bufn;
        tma::mbar_expect_tx(bar + s, gbytes + (cok ? sbytes : 0u));
        tma::bulk_g2s(bs, in + ((long long)bb * nrows + row0) * L * nk, gbytes, bar + s);
        if (cok) tma::bulk_g2s(bs + gridn, S + (long long)c * nvox + row0 * N3, sbytes, bar + s);
    };

    // pass-2 role, fixed across the coils of a unit: line l2, FFT index q1
    const imap::LinePos r2 = imap::pos_fastest(tid, A);
    const int q12 = r2.p, l2 = r2.l;
    const bool p2 = tid < NL * A;
    const imap::UnitLine ul2 = imap::unit_line_split(l2, nk);
    const int rr2 = ul2.rr, kk2 = ul2.kk;
    auto ovox = [&](int q2) {   // output voxel of FFT index q1 + A q2 (>= N3 when cropped away)
        int o = q12 + A * q2 + h;
        return o >= L ? o - L : o;
    };
    float2 acc[B];
    StaticFor<0, B>::run([&](auto qc) { acc[decltype(qc)::value] = make_float2(0.f, 0.f); });

    if (tid == 0 && nsteps > 0) issue(0, 0);
    bool pending[2] = {nsteps > 0, false};     // meaningful in thread 0
    for (long long k = 0; k < nsteps; ++k) {
        const int s = (int)(k & 1);
        if (tid == 0 && k + 1 < nsteps) {
            issue(k + 1, s ^ 1);
            pending[s ^ 1] = true;
        }
        const bool ok = tma::mbar_wait(bar + s, (uint32_t)(k >> 1) & 1u, status);
        if (tid == 0) pending[s] = !ok;
        if (!__syncthreads_and(ok)) {
            // a copy did not land within the limit: let the ones still in flight finish
            // (bounded) before the shared memory goes away
            if (tid == 0)
                for (int q = 0; q < 2; ++q)
                    if (pending[q]) tma::mbar_wait(bar + q, (uint32_t)((k + (q != s)) >> 1) & 1u, status);
            __syncthreads();
            return;
        }
        const long long row0 = ((long long)blockIdx.x + (k / Bc) * gridDim.x) * R;
        const int bb = (int)(k % Bc);
        const int nr = (int)(nrows - row0 < R ? nrows - row0 : R);
        const int c = coil_idx[bb];
        const bool cok = c >= 0 && c < g.C;
        if (!cok && tid == 0 && status) atomicCAS(status, 0, SDP_ERR_BOUNDS);
        const float2* gs = buf0 + s * bufn;
        const float2* Ss = gs + gridn;
        if (tid < NL * B) {
            const imap::LinePos r1 = imap::line_fastest(tid, NL);
            const int l1 = r1.l, b1 = r1.p;
            const imap::UnitLine ul = imap::unit_line_split(l1, nk);
            const int rr = ul.rr, kk = ul.kk;
            float2 u[A];
            StaticFor<0, A>::run([&](auto ac) {
                constexpr int a = decltype(ac)::value;
                u[a] = rr < nr ? gs[imap::line_elem(rr, L, B * a + b1, nk, kk)] : make_float2(0.f, 0.f);
            });
            RegDft<A, true>::run(u);
            StaticFor<0, A>::run([&](auto qc) {
                constexpr int q1 = decltype(qc)::value;
                Y[l1 * LP + q1 * B + b1] = q1 == 0 ? u[q1] : cmul(u[q1], twiddle(tw, b1 * q1, true));
            });
        }
        __syncthreads();
        if (p2 && rr2 < nr && cok) {
            float2 z[B];
            StaticFor<0, B>::run([&](auto bc) {
                constexpr int b = decltype(bc)::value;
                z[b] = Y[l2 * LP + q12 * B + b];
            });
            RegDft<B, true>::run(z);
            const float2* Sr = Ss + (size_t)rr2 * N3;
            StaticFor<0, B>::run([&](auto qc) {
                constexpr int q2 = decltype(qc)::value;
                const int o = ovox(q2);
                if (o < N3) {
                    float2 sv = Sr[o];
                    sv.y = -sv.y;
                    acc[q2] = cadd(acc[q2], cmul(sv, z[q2]));
                }
            });
        }
        if (bb == Bc - 1) {
            // the unit's last coil: scale by 1 / psi_hat, store, start the next unit's sums
            if (p2 && rr2 < nr) {
                const long long row = row0 + rr2;
                const int i1 = (int)(row / N2), i2 = (int)(row - (long long)i1 * N2);
                const float d12 = d1[i1] * d2[i2];
                float2* dst = out + (long long)(k0 + kk2) * nvox + row * N3;
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
            StaticFor<0, B>::run([&](auto qc) { acc[decltype(qc)::value] = make_float2(0.f, 0.f); });
        }
        __syncthreads();   // Y and buffer s are free for the next pass 1 and step k + 2's copies
    }
}

template <class F>
bool with_len_staged(int L, F&& f) {
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

}  // namespace

// The staged prologue needs: a two-pass length, even N3 (16-byte aligned row
// runs), 16-byte aligned x and S, one row's channels within a unit, and shared
// memory for the two buffers.
bool fft2_prologue_staged_ok(const Geo& g, const FftAxis& ax, const float2* x, const float2* S, int nk) {
    if (g.N[2] % 2 || (reinterpret_cast<uintptr_t>(x) & 15) || (reinterpret_cast<uintptr_t>(S) & 15)) return false;
    bool ok = false;
    with_len_staged(ax.L, [&](auto sh) {
        using Sh = decltype(sh);
        ok = staged_rows<Sh::a, Sh::b>(nk) >= 1 && staged_smem<Sh::a, Sh::b>(nk, g.N[2]) <= 200 * 1024;
    });
    return ok;
}

cudaError_t launch_fft2_prologue_staged(const Geo& g, const FftAxis& ax, const float2* x, const float2* S,
                                        const int* coil_idx, int B, int k0, int nk, const float* dinv1,
                                        const float* dinv2, const float* dinv3, float2* out, int* status,
                                        cudaStream_t st) {
    cudaError_t err = cudaErrorNotSupported;
    with_len_staged(ax.L, [&](auto sh) {
        using Sh = decltype(sh);
        auto kern = fft2_prologue_staged_kernel<Sh::a, Sh::b>;
        const size_t smem = staged_smem<Sh::a, Sh::b>(nk, g.N[2]);
        const int R = staged_rows<Sh::a, Sh::b>(nk);
        if (R < 1) return;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
            err = cudaGetLastError();
            return;
        }
        int per_sm = 0, dev = 0, nsm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, staged_threads<Sh::a, Sh::b>(), smem) !=
                cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) {
            err = cudaErrorInvalidDevice;
            return;
        }
        const long long nrows = (long long)g.N[0] * g.N[1];
        const long long nunits = (nrows + R - 1) / R * B;
        const long long grid = std::min<long long>(nunits, (long long)nsm * per_sm);
        if (grid < 1) {
            err = cudaSuccess;
            return;
        }
        kern<<<(unsigned)grid, staged_threads<Sh::a, Sh::b>(), smem, st>>>(g, ax.tw, x, S, coil_idx, B, k0, nk, dinv1,
                                                                           dinv2, dinv3, out, status);
        err = cudaGetLastError();
    });
    return err;
}

// The staged epilogue needs: a two-pass length, even N3, 16-byte aligned grid and
// coil maps, one row's channels within a unit, and shared memory for the buffers.
bool fft2_epilogue_staged_ok(const Geo& g, const FftAxis& ax, const float2* in, const float2* S, int nk) {
    if (g.N[2] % 2 || (reinterpret_cast<uintptr_t>(in) & 15) || (reinterpret_cast<uintptr_t>(S) & 15)) return false;
    bool ok = false;
    with_len_staged(ax.L, [&](auto sh) {
        using Sh = decltype(sh);
        ok = staged_rows<Sh::a, Sh::b>(nk) >= 1 && staged_epi_smem<Sh::a, Sh::b>(nk, g.N[2]) <= 200 * 1024;
    });
    return ok;
}

cudaError_t launch_fft2_epilogue_staged(const Geo& g, const FftAxis& ax, const float2* in, const float2* S,
                                        const int* coil_idx, int B, int k0, int nk, const float* dinv1,
                                        const float* dinv2, const float* dinv3, float2* out, int accumulate,
                                        int* status, cudaStream_t st) {
    cudaError_t err = cudaErrorNotSupported;
    with_len_staged(ax.L, [&](auto sh) {
        using Sh = decltype(sh);
        auto kern = fft2_epilogue_staged_kernel<Sh::a, Sh::b>;
        const size_t smem = staged_epi_smem<Sh::a, Sh::b>(nk, g.N[2]);
        const int R = staged_rows<Sh::a, Sh::b>(nk);
        if (R < 1) return;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
            err = cudaGetLastError();
            return;
        }
        int per_sm = 0, dev = 0, nsm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, staged_threads<Sh::a, Sh::b>(), smem) !=
                cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) {
            err = cudaErrorInvalidDevice;
            return;
        }
        const long long nrows = (long long)g.N[0] * g.N[1];
        const long long nunits = (nrows + R - 1) / R;
        const long long grid = std::min<long long>(nunits, (long long)nsm * per_sm);
        if (grid < 1) {
            err = cudaSuccess;
            return;
        }
        kern<<<(unsigned)grid, staged_threads<Sh::a, Sh::b>(), smem, st>>>(g, ax.tw, in, S, coil_idx, B, k0, nk, dinv1,
                                                                           dinv2, dinv3, out, accumulate, status);
        err = cudaGetLastError();
    });
    return err;
}

}  // namespace sdp
