// Residual and loss without any device allocation.
//
// Some callers cannot call cudaMalloc at all: code running where the device
// memory is owned by someone else (a host framework whose allocator must see
// every byte, a process under a hard memory cap, or work recorded while the
// caller forbids new allocations).  They cannot create a plan, because a plan
// allocates.  sdp_residual_loss_noalloc gives them the data-consistency
// residual and loss with no plan: its scratch (one float64 partial sum per
// chunk of 2^16 residual entries and a completion counter) lives in a
// file-scope __device__ array that the library image carries, at most
// SDP_NOALLOC_MAX_ELEMS residual entries per call.
//
// That array exists once per device that loads the library, for the life of
// the process, and every call on that device shares it: calls that overlap on
// the GPU (different streams, or different host threads) race on it and must
// be serialised by the caller.  The counter is cleared by each call before its
// kernel runs; the partial sums are always fully rewritten.
#include <mutex>

#include "sdp_internal.cuh"

namespace sdp {
namespace {

constexpr int kThreads = 256;
constexpr long long kChunk = 1LL << 16;
constexpr int kMaxChunks = 4096;           // 4096 chunks x 2^16 = 2^28 entries
constexpr int kMaxDevices = 64;

// The fixed scratch must hold one partial per chunk of the largest accepted call.
static_assert((long long)kMaxChunks * kChunk >= SDP_NOALLOC_MAX_ELEMS,
              "noalloc scratch holds fewer chunk partials than SDP_NOALLOC_MAX_ELEMS needs");

struct NoAllocScratch {
    double partials[kMaxChunks];
    unsigned int counter;
};

// 32 KB + 256 B per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch) + 256];

std::mutex g_mu;
NoAllocScratch* g_ptr[kMaxDevices] = {};

// One block per chunk of the flattened [B][J] residual; each block reduces its
// chunk in a fixed order, the last block to finish sums the chunk partials in
// chunk order.  A thread takes the entries e0 + tid + 256 i of its chunk and
// adds their |r|^2 in float32 four at a time, then the group sum into a float64
// accumulator (the FP64 pipe of this part is far too narrow for per-entry
// float64 work).  Its row b and offset j are found once with one division and
// then advanced by the stride; the division runs again only when j passes the
// end of a row.
__global__ void __launch_bounds__(kThreads) residual_loss_chunked_kernel(
    const float2* yhat, const float2* __restrict__ ymeas, const int* __restrict__ meas_idx, long long J,
    int nrows, long long total, float2* r2, NoAllocScratch* scr, float* __restrict__ loss) {
    __shared__ double red[kThreads / 32];
    __shared__ bool s_last;
    const long long e0 = (long long)blockIdx.x * kChunk;
    const long long e1 = e0 + kChunk < total ? e0 + kChunk : total;
    long long e = e0 + threadIdx.x;
    long long b = e / J;
    long long j = e - b * J;
    double acc = 0.0;
    float part = 0.f;
    int nin = 0;
    for (; e < e1; e += kThreads) {
        const int row = __ldg(meas_idx + b);
        float2 r = make_float2(0.f, 0.f);
        if (row >= 0 && row < nrows) {
            const float2 h = yhat[e];
            const float2 m = __ldg(ymeas + (long long)row * J + j);
            r = make_float2(h.x - m.x, h.y - m.y);
        }
        part = fmaf(r.x, r.x, fmaf(r.y, r.y, part));
        if (++nin == 4) {
            acc += (double)part;
            part = 0.f;
            nin = 0;
        }
        r2[e] = make_float2(2.f * r.x, 2.f * r.y);
        j += kThreads;
        if (j >= J) {
            b += j / J;
            j %= J;
        }
    }
    acc += (double)part;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += red[w];
        scr->partials[blockIdx.x] = s;
        __threadfence();
        const unsigned prev = atomicAdd(&scr->counter, 1u);
        s_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        double s = 0.0;
        for (unsigned i = 0; i < gridDim.x; ++i) s += __ldcg(scr->partials + i);
        *loss = (float)s;
        scr->counter = 0u;
    }
}

// Device address of this device's scratch array, looked up once per device
// (with that device current) and cached.
int scratch_for_current_device(NoAllocScratch** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return SDP_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return SDP_ERR_CUDA;
        }
        g_ptr[dev] = reinterpret_cast<NoAllocScratch*>(p);
    }
    *out = g_ptr[dev];
    return SDP_OK;
}

}  // namespace
}  // namespace sdp

extern "C" int sdp_residual_loss_noalloc(const void* yhat, const void* y_meas, int32_t n_meas_rows,
                                         const int32_t* meas_idx, int32_t B, int64_t J, void* r2, float* loss,
                                         void* stream) {
    using namespace sdp;
    if (!yhat || !y_meas || !meas_idx || !r2 || !loss) return SDP_ERR_INVALID_ARG;
    if (B < 1 || J < 1 || n_meas_rows < 1) return SDP_ERR_INVALID_ARG;
    const long long total = (long long)B * J;
    if (total > SDP_NOALLOC_MAX_ELEMS) return SDP_ERR_INVALID_ARG;
    NoAllocScratch* scr = nullptr;
    const int rc = scratch_for_current_device(&scr);
    if (rc != SDP_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(&scr->counter, 0, sizeof(unsigned int), st) != cudaSuccess) {
        cudaGetLastError();
        return SDP_ERR_CUDA;
    }
    const unsigned nblk = (unsigned)((total + kChunk - 1) / kChunk);
    residual_loss_chunked_kernel<<<nblk, kThreads, 0, st>>>(
        static_cast<const float2*>(yhat), static_cast<const float2*>(y_meas), meas_idx, (long long)J, n_meas_rows,
        total, static_cast<float2*>(r2), scr, loss);
    if (cudaGetLastError() != cudaSuccess) return SDP_ERR_CUDA;
    return SDP_OK;
}
