// Several applications of the operator (several plans: volumes of different
// matrix sizes, uneven coil minibatches) in ONE launch per stage (StoDIP Eq. 3
// for several reconstructions at once).
//
// A batched forward is four launches whatever the number of items: the fused
// prologue + axis-3 FFT, the axis-2 FFT, the axis-1 FFT and the interpolation;
// a batched adjoint is the spread, the inverse axis-1 and axis-2 FFTs and the
// fused axis-3 FFT + epilogue.  Each launch covers the units of work of every
// item: an item's units are a contiguous range of the launch's unit index
// (the host passes the prefix sums), a CTA finds its item with a short scan of
// that table, and runs the same per-unit body the single-plan kernels run
// (fft2_impl.cuh, interp_impl.cuh, spread_impl.cuh), on that item's pointers
// and sizes.  The FFT kernels switch on the item's axis length, so items of
// different grid sizes share a launch; lines (or columns) per CTA follow from
// the length so that every shape fills the CTA's threads.  The interpolation
// is persistent (its warps walk the concatenated, bin-sorted samples of all
// items); the other stages launch one CTA per unit and let the hardware
// scheduler balance them.  Stage order is kernel order on the stream: no
// CTA waits for another.
//
// Items that share a plan use disjoint coil slices of its workspace, so they
// run in the same launches as long as their minibatches fit the plan's
// max_batch together (the host splits the batch into waves otherwise).
#include <algorithm>

#include "batch.cuh"
#include "fft2_impl.cuh"

namespace sdp {
namespace {

constexpr int kFusedThreads = 128;     // fused axis-3 kernels
constexpr int kStridedThreads = 256;   // strided passes

// Compile-time (A, B) of every length with a two-pass kernel, and the switch over them.
template <class F>
__device__ __forceinline__ void with_len(int L, F&& f) {
    using std::integral_constant;
    switch (L) {
        case 48: f(integral_constant<int, 8>{}, integral_constant<int, 6>{}); break;
        case 64: f(integral_constant<int, 8>{}, integral_constant<int, 8>{}); break;
        case 80: f(integral_constant<int, 10>{}, integral_constant<int, 8>{}); break;
        case 96: f(integral_constant<int, 12>{}, integral_constant<int, 8>{}); break;
        case 100: f(integral_constant<int, 10>{}, integral_constant<int, 10>{}); break;
        case 120: f(integral_constant<int, 12>{}, integral_constant<int, 10>{}); break;
        case 128: f(integral_constant<int, 16>{}, integral_constant<int, 8>{}); break;
        case 160: f(integral_constant<int, 16>{}, integral_constant<int, 10>{}); break;
        case 200: f(integral_constant<int, 20>{}, integral_constant<int, 10>{}); break;
        case 240: f(integral_constant<int, 16>{}, integral_constant<int, 15>{}); break;
        case 250: f(integral_constant<int, 25>{}, integral_constant<int, 10>{}); break;
        case 256: f(integral_constant<int, 16>{}, integral_constant<int, 16>{}); break;
        default: break;
    }
}

constexpr int kLenA[] = {8, 8, 10, 12, 10, 12, 16, 16, 20, 16, 25, 16};
constexpr int kLenB[] = {6, 8, 8, 8, 10, 10, 8, 10, 10, 15, 10, 16};

__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }

// Lines (or columns) per CTA of a length with NT threads: as many as fill them.
template <int A, int B, int NT>
__host__ __device__ constexpr int lines_for() { return NT / cmax(A, B); }

// Shared memory (float2 elements) the largest shape needs: tw[L] + Y.
constexpr int fused_smem() {
    int m = 0;
    for (int i = 0; i < 12; ++i) {
        const int L = kLenA[i] * kLenB[i], nl = kFusedThreads / cmax(kLenA[i], kLenB[i]);
        m = cmax(m, L + nl * (L + 1));
    }
    return m;
}
constexpr int strided_smem() {
    int m = 0;
    for (int i = 0; i < 12; ++i) {
        const int L = kLenA[i] * kLenB[i], nl = kStridedThreads / cmax(kLenA[i], kLenB[i]);
        m = cmax(m, L + nl * L);
    }
    return m;
}
constexpr int kFusedSmem = fused_smem();
constexpr int kStridedSmem = strided_smem();
static_assert(kFusedSmem * 8 <= 48 * 1024 && kStridedSmem * 8 <= 48 * 1024, "static shared memory of the batch kernels");

__device__ __forceinline__ int find_item(const MvUnits& u, long long unit) {
    int i = 0;
    while (i + 1 < u.n && unit >= u.start[i + 1]) ++i;
    return i;
}

// The per-length units are separate (not inlined) functions: each gets its own
// register allocation, so a launch's register count is that of its largest
// shape instead of the union of all shapes' live values.

// ---- forward: prologue + axis 3 ----
template <int A, int B>
__device__ __noinline__ void prologue_unit(float2* smem, const MvItem& it, long long blk) {
    constexpr int NL = lines_for<A, B, kFusedThreads>();
    fft2_prologue_body<A, B, NL>(smem, smem + A * B, it.g, it.tw[2], it.x, it.S, it.coil_idx, it.B, 0, it.g.K,
                                 it.d[0], it.d[1], it.d[2], it.bufA, it.status, blk);
}

__global__ void __launch_bounds__(kFusedThreads, 7) mv_prologue_kernel(const MvArgs a, const MvUnits u) {
    __shared__ float2 smem[kFusedSmem];
    for (long long unit = blockIdx.x; unit < u.start[u.n]; unit += gridDim.x) {
        const int i = find_item(u, unit);
        const MvItem& it = a.it[i];
        const long long blk = unit - u.start[i];
        with_len(it.L[2], [&](auto ac, auto bc) { prologue_unit<decltype(ac)::value, decltype(bc)::value>(smem, it, blk); });
    }
}

// ---- strided passes (axis 1 or 2, forward or inverse) ----
template <int A, int B, bool INV>
__device__ __noinline__ void strided_unit(float2* smem, const MvItem& it, int axis, long long blk) {
    constexpr int NL = lines_for<A, B, kStridedThreads>();
    const MvPass& ps = it.pass[axis];
    const long long ncolblk = (ps.inner + NL - 1) / NL;
    fft2_strided_body<A, B, NL, INV>(smem, smem + A * B, ps.in, ps.out, it.tw[axis], ps.n_in, ps.in_centred,
                                     ps.n_out, ps.out_centred, ps.inner, ncolblk, blk);
}

template <bool INV>
__global__ void __launch_bounds__(kStridedThreads, 4) mv_strided_kernel(const MvArgs a, const MvUnits u, int axis) {
    __shared__ float2 smem[kStridedSmem];
    for (long long unit = blockIdx.x; unit < u.start[u.n]; unit += gridDim.x) {
        const int i = find_item(u, unit);
        const MvItem& it = a.it[i];
        const long long blk = unit - u.start[i];
        with_len(it.L[axis], [&](auto ac, auto bc) {
            strided_unit<decltype(ac)::value, decltype(bc)::value, INV>(smem, it, axis, blk);
        });
    }
}

// ---- adjoint: axis 3 + epilogue ----
template <int A, int B>
__device__ __noinline__ void epilogue_unit(float2* smem, const MvItem& it, long long blk) {
    constexpr int NL = lines_for<A, B, kFusedThreads>();
    fft2_epilogue_body<A, B, NL>(smem, smem + A * B, it.g, it.tw[2], it.bufA, it.S, it.coil_idx, it.B, 0, it.g.K,
                                 it.d[0], it.d[1], it.d[2], it.x, it.accumulate, it.status, blk);
}

__global__ void __launch_bounds__(kFusedThreads, 4) mv_epilogue_kernel(const MvArgs a, const MvUnits u) {
    __shared__ float2 smem[kFusedSmem];
    for (long long unit = blockIdx.x; unit < u.start[u.n]; unit += gridDim.x) {
        const int i = find_item(u, unit);
        const MvItem& it = a.it[i];
        const long long blk = unit - u.start[i];
        with_len(it.L[2], [&](auto ac, auto bc) { epilogue_unit<decltype(ac)::value, decltype(bc)::value>(smem, it, blk); });
    }
}

unsigned grid_of(const MvUnits& u) {
    const long long n = u.start[u.n];
    return (unsigned)std::min<long long>(n, 0x7fffffffLL);
}

}  // namespace

bool mv_length_supported(int L) {
    for (int i = 0; i < 12; ++i)
        if (kLenA[i] * kLenB[i] == L) return true;
    return false;
}

long long mv_fused_lines(int L) {
    for (int i = 0; i < 12; ++i)
        if (kLenA[i] * kLenB[i] == L) return kFusedThreads / cmax(kLenA[i], kLenB[i]);
    return 0;
}

long long mv_strided_cols(int L) {
    for (int i = 0; i < 12; ++i)
        if (kLenA[i] * kLenB[i] == L) return kStridedThreads / cmax(kLenA[i], kLenB[i]);
    return 0;
}

cudaError_t launch_mv_prologue(const MvArgs& a, const MvUnits& u, cudaStream_t st) {
    if (u.start[u.n] == 0) return cudaSuccess;
    mv_prologue_kernel<<<grid_of(u), kFusedThreads, 0, st>>>(a, u);
    return cudaGetLastError();
}

cudaError_t launch_mv_strided(const MvArgs& a, const MvUnits& u, int axis, int inverse, cudaStream_t st) {
    if (u.start[u.n] == 0) return cudaSuccess;
    if (inverse)
        mv_strided_kernel<true><<<grid_of(u), kStridedThreads, 0, st>>>(a, u, axis);
    else
        mv_strided_kernel<false><<<grid_of(u), kStridedThreads, 0, st>>>(a, u, axis);
    return cudaGetLastError();
}

cudaError_t launch_mv_epilogue(const MvArgs& a, const MvUnits& u, cudaStream_t st) {
    if (u.start[u.n] == 0) return cudaSuccess;
    mv_epilogue_kernel<<<grid_of(u), kFusedThreads, 0, st>>>(a, u);
    return cudaGetLastError();
}

}  // namespace sdp
