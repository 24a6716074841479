// MRF dictionary matching (StoDIP, Sec. 2 after Eq. 1; Ma et al. 2013,
// McGivney et al. 2014): for every voxel v of the TSMI and every compressed
// atom d_p,  idx_v = argmax_p |d_p^H x_v| / ||d_p||,  PD_v = d_idx^H x_v / ||d_idx||^2.
//
// Three kernels per match:
//  1. dm_prep_voxels: x_v / ||x_v|| to fp16, written in the tcgen05 shared-memory
//     tile layout (128 voxels x 16 k-values per 4 KB tile, 8x8 core matrices,
//     K-major, no swizzle); row v holds (Re x_v, Im x_v, 0 ...).
//  2. dm_score_kernel: a persistent tcgen05 GEMM.  One CTA per SM walks pairs
//     of voxel tiles; for each pair it streams the fp16 atom tiles (64 atoms =
//     128 rows (Re-column, Im-column) each) through a shared-memory ring with
//     bulk copies, two threads (one per voxel tile) issue M=128 x N=128 x K=16
//     MMAs into fp32 accumulators in
//     tensor memory (two buffers x two voxel tiles x 128 columns = all 512
//     columns), and sixteen epilogue warps read the accumulators with
//     tcgen05.ld (one warp per voxel tile, 64-column half and lane quarter),
//     form |d^H x|^2 =
//     Re^2 + Im^2 of every (voxel, atom) with packed f32x2 arithmetic and keep,
//     per voxel and half, the 32-atom chunk with the largest score (first
//     chunk on ties).  The two halves are merged by the refine pass, so the
//     epilogue warps never wait on each other.
//  3. dm_refine: a warp per 4 voxels takes, for each, the better of its two half results
//     (lower chunk on ties), recomputes the 32 inner products of that
//     chunk in float32 from the float32 inputs and takes the argmax (lowest
//     atom on ties) and PD.
// Every wait on an mbarrier is bounded (about one second); a wait that gives
// up sets the status word to SDP_ERR_TIMEOUT, the block stops issuing work,
// drains what it has in flight and frees its tensor memory.
#include <algorithm>
#include <atomic>
#include <new>

#include <cuda_fp16.h>

#include "../../include/stodip_dm.h"
#include "sdp_internal.cuh"

namespace sdp {
namespace {

constexpr int BM = 128;                     // voxels per tile = tensor-memory lanes
constexpr int VT = 2;                       // voxel tiles per step of a CTA
constexpr int BN = 128;                     // accumulator columns per atom tile (64 atoms x Re, Im)
constexpr int ATOMS_PER_TILE = BN / 2;
constexpr int NACC = 2;                     // accumulator buffers (each: VT voxel tiles x BN columns)
constexpr int CHUNK = 32;                   // atoms per tcgen05.ld of 64 columns
constexpr int NB = 8;                       // atom-tile ring stages
constexpr int kEpiWarps = 16;               // 2 voxel tiles x 2 column halves x 4 lane quarters
constexpr int kThreadsG = 128 + 32 * kEpiWarps;
constexpr uint32_t kTmemCols = 512;         // 2 buffers x 2 voxel tiles x 128 columns
constexpr unsigned long long kTimeoutNs = 1000000000ull;   // default limit of every mbarrier wait
constexpr int kMinSmem = 120 * 1024;        // keeps one CTA (and one tensor-memory owner) per SM

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) from
// global to shared memory, completing as transaction bytes on `bar`.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of tcgen05 for a K-major, unswizzled tile:
// start address, leading byte offset (between the 8x16-byte core matrices
// adjacent along K), stride byte offset (between 8-row groups), version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// D[tmem] (+)= A[smem] * B[smem]^T, fp16 inputs, fp32 accumulator.
__device__ __forceinline__ void tc_mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

// Arrive on `bar` once every tcgen05 operation this thread issued so far has completed.
__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld_x32(uint32_t taddr, float (&v)[32]) {
    uint32_t* r = reinterpret_cast<uint32_t*>(v);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Bounded wait for the completion of the phase of `bar` with parity `parity`.
// Gives up after `limit_ns` of %globaltimer (recording SDP_ERR_TIMEOUT and
// raising the block's abort flag), or at once when the abort flag is up and
// `honour_abort`.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* status,
                                          bool honour_abort, unsigned long long limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = gtimer();
    while (!mbar_try_wait(bar, parity)) {
        if (honour_abort && *abort_flag) return false;
        if (gtimer() - t0 > limit_ns) {
            *abort_flag = 1;
            atomicCAS(status, 0, SDP_ERR_TIMEOUT);
            return false;
        }
    }
    return true;
}

// ---------------------------------------------------------------------------
// fp16 tiles in the tcgen05 layout: a tile is 128 rows x 16*KS k-values; the
// 8x8 core matrix (8 rows x 16 bytes) of row group r/8 and k-chunk c sits at
// (r/8) * KS*256 + c * 128, its row r%8 at + (r%8) * 16.  So the leading byte
// offset (next core matrix along K) is 128 and the stride byte offset (next
// 8-row group) is KS*256.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t tile_off(int r, int c, int KS) {
    return (uint32_t)((r >> 3) * (KS * 256) + c * 128 + (r & 7) * 16);
}

__device__ __forceinline__ void store_row(uint8_t* tile, int r, int KS, const float* e) {
    // e: the row's 16*KS values
    for (int c = 0; c < 2 * KS; ++c) {
        __align__(16) __half h[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) h[j] = __float2half_rn(e[c * 8 + j]);
        *reinterpret_cast<uint4*>(tile + tile_off(r, c, KS)) = *reinterpret_cast<const uint4*>(h);
    }
}

// Atoms: 1/||d_p|| (0 for a zero atom), the unit atoms in float32, and two fp16
// rows per atom in its tile: the Re-column (Re d, Im d) and the Im-column
// (-Im d, Re d), so that row . (Re x, Im x) = Re(d^H x) and Im(d^H x).  Within
// a tile of 64 atoms the rows of atoms 2q and 2q+1 are ordered
// Re(2q), Re(2q+1), Im(2q), Im(2q+1) (rows 4q .. 4q+3).  Padding atoms are zero.
__global__ void dm_prep_atoms(const float2* __restrict__ atoms, long long P, int K, int KS, long long npad,
                              float2* __restrict__ dhat, float* __restrict__ inv_norm, uint8_t* __restrict__ bh) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npad) return;
    float2 d[kMaxK];
    double ss = 0.0;
    for (int k = 0; k < K; ++k) {
        d[k] = p < P ? atoms[p * K + k] : make_float2(0.f, 0.f);
        ss += (double)d[k].x * d[k].x + (double)d[k].y * d[k].y;
    }
    const float inv = ss > 0.0 ? (float)(1.0 / sqrt(ss)) : 0.f;
    if (p < P) {
        inv_norm[p] = inv;
        for (int k = 0; k < K; ++k) dhat[p * K + k] = make_float2(d[k].x * inv, d[k].y * inv);
    }
    float re[32], im[32];
    for (int e = 0; e < 16 * KS; ++e) {
        re[e] = e < K ? d[e].x * inv : (e < 2 * K ? d[e - K].y * inv : 0.f);
        im[e] = e < K ? -d[e].y * inv : (e < 2 * K ? d[e - K].x * inv : 0.f);
    }
    const int a = (int)(p % ATOMS_PER_TILE), q = a >> 1, odd = a & 1;
    uint8_t* tile = bh + (p / ATOMS_PER_TILE) * (long long)(KS * 4096);
    store_row(tile, 4 * q + odd, KS, re);
    store_row(tile, 4 * q + 2 + odd, KS, im);
}

// Voxels: x_v / ||x_v|| as one fp16 row (Re x_v, Im x_v, 0 ...); rows past nvox
// are zero.  The norm is taken after scaling by the largest component, so it
// neither overflows nor underflows in float32.
__global__ void dm_prep_voxels(const float2* __restrict__ x, long long nvox, int K, int KS, long long nrows,
                               uint8_t* __restrict__ xh) {
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nrows) return;
    float2 xv[kMaxK];
    float m = 0.f;
    for (int k = 0; k < K; ++k) {
        xv[k] = v < nvox ? __ldg(x + k * nvox + v) : make_float2(0.f, 0.f);
        m = fmaxf(m, fmaxf(fabsf(xv[k].x), fabsf(xv[k].y)));
    }
    float inv = 0.f;
    if (m > 0.f) {
        const float im = 1.f / m;
        float ss = 0.f;
        for (int k = 0; k < K; ++k) ss += (xv[k].x * im) * (xv[k].x * im) + (xv[k].y * im) * (xv[k].y * im);
        inv = im * rsqrtf(ss);
    }
    float e[32];
    for (int j = 0; j < 16 * KS; ++j) e[j] = j < K ? xv[j].x * inv : (j < 2 * K ? xv[j - K].y * inv : 0.f);
    store_row(xh + (v / BM) * (long long)(KS * 4096), (int)(v % BM), KS, e);
}

// Refine: a warp resolves RV voxels.  For voxel j the warp takes the better of
// its two half results (lower chunk on ties); lane l scores atom
// p = 32 * chunk + l in float32, and the warp takes the argmax (lowest atom on
// ties) and PD = (d_p/||d_p||)^H x / ||d_p||.  The RV voxels' loads are
// independent and issued together, so a warp has several round trips in flight.
constexpr int RV = 4;

__global__ void __launch_bounds__(256) dm_refine(const float2* __restrict__ x, long long nvox, int K,
                                                 const float* __restrict__ best_score,
                                                 const int* __restrict__ best_chunk,
                                                 const float2* __restrict__ dhat, const float* __restrict__ inv_norm,
                                                 long long P, int nchunk, const float2* __restrict__ params,
                                                 int* __restrict__ idx, float2* __restrict__ pd,
                                                 float2* __restrict__ qmap) {
    const int lane = threadIdx.x & 31;
    const long long vb = ((long long)blockIdx.x * 8 + (threadIdx.x >> 5)) * RV;
    if (vb >= nvox) return;                                       // uniform over the warp
    int cl = 0;                                                   // lane j < RV: chunk of voxel vb + j
    if (lane < RV && vb + lane < nvox) {
        const long long v = vb + lane;
        const float s0 = __ldg(best_score + v), s1 = __ldg(best_score + nvox + v);
        const int c0 = __ldg(best_chunk + v), c1 = __ldg(best_chunk + nvox + v);
        cl = (s1 > s0 || (s1 == s0 && c1 < c0)) ? c1 : c0;
        // after a timed-out score kernel the chunk may be stale: keep every load in range
        cl = min(max(cl, 0), nchunk - 1);
    }
    long long p[RV];
    float2 s[RV];
#pragma unroll
    for (int j = 0; j < RV; ++j) {
        p[j] = (long long)__shfl_sync(0xffffffffu, cl, j) * CHUNK + lane;
        s[j] = make_float2(0.f, 0.f);
    }
    for (int k = 0; k < K; ++k) {
#pragma unroll
        for (int j = 0; j < RV; ++j) {
            if (vb + j < nvox && p[j] < P) {
                const float2 xk = __ldg(x + k * nvox + vb + j);
                const float2 d = __ldg(dhat + p[j] * K + k);
                s[j].x += d.x * xk.x + d.y * xk.y;
                s[j].y += d.x * xk.y - d.y * xk.x;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < RV; ++j) {
        float best = p[j] < P ? s[j].x * s[j].x + s[j].y * s[j].y : -1.f;
        int bl = lane;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int ol = __shfl_xor_sync(0xffffffffu, bl, o);
            if (ov > best || (ov == best && ol < bl)) {
                best = ov;
                bl = ol;
            }
        }
        const long long v = vb + j;
        if (lane == bl && v < nvox) {
            if (p[j] < P) {
                const float in = __ldg(inv_norm + p[j]);
                idx[v] = (int)p[j];
                pd[v] = make_float2(s[j].x * in, s[j].y * in);
                if (qmap) qmap[v] = __ldg(params + p[j]);
            } else {                   // a chunk past the last atom (not chosen by the score kernel)
                idx[v] = 0;
                pd[v] = make_float2(0.f, 0.f);
                if (qmap) qmap[v] = __ldg(params);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// The tcgen05 score kernel
// ---------------------------------------------------------------------------
struct GemmArgs {
    const uint8_t* xh;      // voxel tiles (2 * npairs of them)
    const uint8_t* bh;      // atom tiles (ntiles)
    long long nvox;
    int npairs;
    int ntiles;
    float* best_score;      // [2][nvox]: per column half, the best fp16-path score
    int* best_chunk;        // [2][nvox]: and its chunk
    int* status;
    unsigned long long timeout_ns;   // limit of every mbarrier wait
    int withhold_tile;      // test hook: CTA 0 never copies this atom tile of its first step (-1: off)
};

// Largest |d^H x|^2 over the 16 atoms of 32 accumulator columns laid out
// Re(2q), Re(2q+1), Im(2q), Im(2q+1): the squares of an atom pair in one
// packed f32x2 multiply and fused multiply-add, then a three-input max.
__device__ __forceinline__ float half_max(const float (&v)[32]) {
    float m[4] = {0.f, 0.f, 0.f, 0.f};          // four independent running maxima
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        unsigned long long re, im, s2;
        asm("mov.b64 %0, {%1, %2};" : "=l"(re) : "f"(v[4 * q]), "f"(v[4 * q + 1]));
        asm("mov.b64 %0, {%1, %2};" : "=l"(im) : "f"(v[4 * q + 2]), "f"(v[4 * q + 3]));
        asm("mul.rn.f32x2 %0, %1, %1;" : "=l"(s2) : "l"(re));
        asm("fma.rn.f32x2 %0, %1, %1, %2;" : "=l"(s2) : "l"(im), "l"(s2));
        float sa, sb;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(sa), "=f"(sb) : "l"(s2));
        asm("max.f32 %0, %1, %2, %3;" : "=f"(m[q & 3]) : "f"(m[q & 3]), "f"(sa), "f"(sb));
    }
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(m[0]), "f"(m[1]), "f"(m[2]));
    return fmaxf(r, m[3]);
}

template <int KS>
__host__ __device__ constexpr uint32_t tile_bytes() { return KS * 4096u; }

template <int KS>
constexpr int score_smem_bytes() {
    return 1024 + (2 * VT + NB) * (int)tile_bytes<KS>() + (4 + 2 * NB + 2 * VT * NACC + VT) * 8 + 8;
}

// Warp roles: warp 0 lane 0 copies tiles in (bulk copies), lane 0 of warp 1
// (voxel tile 0) and of warp 3 (voxel tile 1) issue the MMAs, each with its own
// accumulator barriers so the two wait/issue/commit chains run side by side,
// warp 2 owns the tensor memory, warps 4..19 are the
// epilogue (warp 4 + 8u + 4h + q reads lanes 32q..32q+31, columns 64h..64h+63
// of voxel tile u).
template <int KS>
__global__ void __launch_bounds__(kThreadsG, 1) dm_score_kernel(GemmArgs g) {
    constexpr uint32_t TB = tile_bytes<KS>();
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = sm;                                  // 2 stages x VT voxel tiles
    uint8_t* sB = sA + 2 * VT * TB;                    // NB atom tiles
    uint64_t* bars = reinterpret_cast<uint64_t*>(sB + NB * TB);
    uint64_t* a_full = bars;                           // [2]
    uint64_t* a_empty = bars + 2;                      // [2]
    uint64_t* b_full = bars + 4;                       // [NB]
    uint64_t* b_empty = bars + 4 + NB;                 // [NB]
    uint64_t* acc_full = bars + 4 + 2 * NB;            // [VT][NACC]
    uint64_t* acc_empty = acc_full + VT * NACC;        // [VT][NACC]
    uint64_t* mma_done = acc_empty + VT * NACC;        // [VT]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + VT);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(smem_u32(a_full + i), 1);
            mbar_init(smem_u32(a_empty + i), VT);               // both MMA threads release a voxel stage
        }
        for (int i = 0; i < VT * NACC; ++i) {
            mbar_init(smem_u32(acc_full + i), 1);
            mbar_init(smem_u32(acc_empty + i), kEpiWarps / VT); // the epilogue warps of one voxel tile
        }
        for (int i = 0; i < NB; ++i) {
            mbar_init(smem_u32(b_full + i), 1);
            mbar_init(smem_u32(b_empty + i), VT);               // both MMA threads release an atom tile
        }
        for (int i = 0; i < VT; ++i) mbar_init(smem_u32(mma_done + i), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int nsteps = (int)blockIdx.x < g.npairs ? (g.npairs - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int ntiles = g.ntiles;

    if (warp == 0) {
        if (lane == 0) {
            long long nb = 0;  // atom tiles issued
            int na = 0;        // voxel-tile pairs issued
            bool ok = true;
            for (int i = 0; i < nsteps && ok; ++i) {
                const int pair = (int)blockIdx.x + i * (int)gridDim.x;
                const int sa = i & 1;
                if (!mbar_wait(smem_u32(a_empty + sa), ((i >> 1) & 1) ^ 1, abort_flag, g.status, true, g.timeout_ns)) break;
                mbar_expect_tx(smem_u32(a_full + sa), VT * TB);
                bulk_g2s(smem_u32(sA + sa * VT * TB), g.xh + (size_t)pair * VT * TB, VT * TB, smem_u32(a_full + sa));
                ++na;
                for (int t = 0; t < ntiles; ++t) {
                    if (i == 0 && t == g.withhold_tile && blockIdx.x == 0) {
                        // test hook: this copy is never issued, so the MMA threads' bounded
                        // wait for it runs out; stop producing and drain what was issued
                        ok = false;
                        break;
                    }
                    const int s = (int)(nb % NB);
                    if (!mbar_wait(smem_u32(b_empty + s), (uint32_t)((nb / NB) & 1) ^ 1u, abort_flag, g.status,
                                   true, g.timeout_ns)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(smem_u32(b_full + s), TB);
                    bulk_g2s(smem_u32(sB + s * TB), g.bh + (size_t)t * TB, TB, smem_u32(b_full + s));
                    ++nb;
                }
            }
            // drain: the last copy into every slot has landed before the block may exit
            for (int s = 0; s < 2; ++s)
                if (na > s) mbar_wait(smem_u32(a_full + s), (uint32_t)(((na - 1 - s) / 2) & 1), abort_flag, g.status, false, g.timeout_ns);
            for (int s = 0; s < NB; ++s)
                if (nb > s)
                    mbar_wait(smem_u32(b_full + s), (uint32_t)(((nb - 1 - s) / NB) & 1), abort_flag, g.status, false, g.timeout_ns);
        }
    } else if (warp == 1 || warp == 3) {
        if (lane == 0) {
            const int u = warp == 1 ? 0 : 1;  // this thread's voxel tile of the pair
            // kind::f16 instruction descriptor: fp32 accumulator, fp16 A and B, both
            // K-major, N = BN, M = BM
            const uint32_t idesc = (1u << 4) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
            uint64_t* accf = acc_full + u * NACC;
            uint64_t* acce = acc_empty + u * NACC;
            long long nb = 0;
            bool ok = true;
            for (int i = 0; i < nsteps && ok; ++i) {
                const int sa = i & 1;
                if (!mbar_wait(smem_u32(a_full + sa), (uint32_t)((i >> 1) & 1), abort_flag, g.status, true, g.timeout_ns)) break;
                tc_fence_after();
                for (int t = 0; t < ntiles; ++t, ++nb) {
                    const int s = (int)(nb % NB);
                    const int b = (int)(nb % NACC);
                    if (!mbar_wait(smem_u32(b_full + s), (uint32_t)((nb / NB) & 1), abort_flag, g.status, true, g.timeout_ns) ||
                        !mbar_wait(smem_u32(acce + b), (uint32_t)((nb / NACC) & 1) ^ 1u, abort_flag, g.status,
                                   true, g.timeout_ns)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tmem + (uint32_t)((b * VT + u) * BN);
#pragma unroll
                    for (int ks = 0; ks < KS; ++ks) {
                        const uint64_t ad = smem_desc(smem_u32(sA + (sa * VT + u) * TB + ks * 256), 128, KS * 256);
                        const uint64_t bd = smem_desc(smem_u32(sB + s * TB + ks * 256), 128, KS * 256);
                        tc_mma_f16(d, ad, bd, idesc, ks > 0 ? 1u : 0u);
                    }
                    tc_commit(smem_u32(b_empty + s));
                    tc_commit(smem_u32(accf + b));
                }
                if (ok) tc_commit(smem_u32(a_empty + sa));
            }
            // every MMA this thread issued has completed before the tensor memory is freed
            tc_commit(smem_u32(mma_done + u));
            mbar_wait(smem_u32(mma_done + u), 0, abort_flag, g.status, false, g.timeout_ns);
        }
    } else if (warp >= 4) {
        const int eg = warp - 4;
        const int quarter = eg & 3;             // tensor-memory lanes 32*quarter .. (= warp % 4)
        const int h = (eg >> 2) & 1;            // column half: atoms 32h .. 32h+31 of each tile
        const int u = eg >> 3;                  // voxel tile of the pair
        const int row = quarter * 32 + lane;
        long long nb = 0;
        bool ok = true;
        for (int i = 0; i < nsteps && ok; ++i) {
            const int pair = (int)blockIdx.x + i * (int)gridDim.x;
            float best = -1.f;
            int bestc = 0;
            for (int t = 0; t < ntiles; ++t, ++nb) {
                const int b = (int)(nb % NACC);
                const bool w = mbar_wait(smem_u32(acc_full + u * NACC + b), (uint32_t)((nb / NACC) & 1), abort_flag, g.status,
                                         true, g.timeout_ns);
                if (!__all_sync(0xffffffffu, w)) {     // warp-uniform: tcgen05.ld is .sync.aligned
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t taddr =
                    tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)((b * VT + u) * BN + h * 64);
                // two 32-column loads: the maximum of the first half is formed while
                // the second half is still on its way from tensor memory
                float va[32], vb[32];
                tmem_ld_x32(taddr, va);
                tmem_wait_ld();
                tmem_ld_x32(taddr + 32, vb);
                const float ma = half_max(va);
                tmem_wait_ld();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(acc_empty + u * NACC + b));
                const float m = fmaxf(ma, half_max(vb));
                if (m > best) {
                    best = m;
                    bestc = 2 * t + h;
                }
            }
            if (!ok) break;
            const long long vox = ((long long)pair * VT + u) * BM + row;
            if (vox < g.nvox) {
                g.best_score[h * g.nvox + vox] = best;
                g.best_chunk[h * g.nvox + vox] = bestc;
            }
        }
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (warp == 2) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

}  // namespace
}  // namespace sdp

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
struct sdp_dm_s {
    long long P = 0, max_vox = 0;
    int K = 0, KS = 0, ntiles = 0, nsm = 0;
    float2* dhat = nullptr;
    float2* params = nullptr;
    float* inv_norm = nullptr;
    uint8_t* bh = nullptr;
    uint8_t* xh = nullptr;
    float* best_score = nullptr;
    int* best = nullptr;
    int* status = nullptr;
    size_t bytes = 0;
    unsigned long long timeout_ns = sdp::kTimeoutNs;
    int withhold_tile = -1;
};

namespace {

using sdp::GemmArgs;

void dm_free(sdp_dm_s* d) {
    if (!d) return;
    cudaFree(d->dhat);
    cudaFree(d->params);
    cudaFree(d->inv_norm);
    cudaFree(d->bh);
    cudaFree(d->xh);
    cudaFree(d->best_score);
    cudaFree(d->best);
    cudaFree(d->status);
    delete d;
}

template <typename T>
bool dm_alloc(sdp_dm_s* d, T** p, size_t n) {
    if (cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    d->bytes += n * sizeof(T);
    return true;
}

long long pairs_for(long long nvox) { return ((nvox + sdp::BM - 1) / sdp::BM + sdp::VT - 1) / sdp::VT; }

}  // namespace

extern "C" {

int sdp_dm_create(sdp_dm_t* out, const void* atoms, const float* params, int64_t P, int32_t K,
                  int64_t max_vox, void* stream) {
    if (!out) return SDP_ERR_INVALID_ARG;
    *out = nullptr;
    if (!atoms || P < 1 || P > (1LL << 24) || K < 1 || K > 16 || max_vox < 1 || max_vox > 2147483647LL)
        return SDP_ERR_INVALID_ARG;
    int dev = 0, major = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return SDP_ERR_CUDA;
    }
    if (major < 10) return SDP_ERR_UNSUPPORTED;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    sdp_dm_s* d = new (std::nothrow) sdp_dm_s;
    if (!d) return SDP_ERR_OOM;
    d->P = P;
    d->K = K;
    d->KS = (2 * K + 15) / 16;
    d->ntiles = (int)((P + sdp::ATOMS_PER_TILE - 1) / sdp::ATOMS_PER_TILE);
    d->max_vox = max_vox;
    d->nsm = nsm;
    const size_t TB = (size_t)d->KS * 4096;
    const long long npairs = pairs_for(max_vox);
    if (!dm_alloc(d, &d->dhat, (size_t)P * K) || !dm_alloc(d, &d->inv_norm, (size_t)P) ||
        !dm_alloc(d, &d->bh, (size_t)d->ntiles * TB) || !dm_alloc(d, &d->xh, (size_t)npairs * sdp::VT * TB) ||
        !dm_alloc(d, &d->best, (size_t)2 * max_vox) || !dm_alloc(d, &d->best_score, (size_t)2 * max_vox) ||
        !dm_alloc(d, &d->status, 1) ||
        (params && !dm_alloc(d, &d->params, (size_t)P))) {
        dm_free(d);
        return SDP_ERR_OOM;
    }
    if (params && cudaMemcpyAsync(d->params, params, (size_t)P * sizeof(float2), cudaMemcpyDeviceToDevice, st) !=
                      cudaSuccess) {
        cudaGetLastError();
        dm_free(d);
        return SDP_ERR_CUDA;
    }
    const long long npad = (long long)d->ntiles * sdp::ATOMS_PER_TILE;
    sdp::dm_prep_atoms<<<(unsigned)((npad + 255) / 256), 256, 0, st>>>(static_cast<const float2*>(atoms), P, K,
                                                                        d->KS, npad, d->dhat, d->inv_norm, d->bh);
    const int smem = d->KS == 1 ? sdp::score_smem_bytes<1>() : sdp::score_smem_bytes<2>();
    const int smem_req = std::max(smem, sdp::kMinSmem);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemsetAsync(d->status, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d->best, 0, (size_t)2 * max_vox * sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d->best_score, 0, (size_t)2 * max_vox * sizeof(float), st);
    if (e == cudaSuccess)
        e = d->KS == 1 ? cudaFuncSetAttribute(sdp::dm_score_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              smem_req)
                       : cudaFuncSetAttribute(sdp::dm_score_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              smem_req);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    sdp::note_launches(1);
    if (e != cudaSuccess) {
        cudaGetLastError();
        dm_free(d);
        return SDP_ERR_CUDA;
    }
    *out = d;
    return SDP_OK;
}

void sdp_dm_destroy(sdp_dm_t dm) { dm_free(dm); }

int sdp_dm_match(sdp_dm_t dm, const void* x, int64_t nvox, int32_t* idx, void* pd, float* qmap, void* stream) {
    if (!dm || nvox < 0 || nvox > dm->max_vox) return SDP_ERR_INVALID_ARG;
    if (nvox == 0) return SDP_OK;
    if (!x || !idx || !pd || (qmap && !dm->params)) return SDP_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const long long npairs = pairs_for(nvox);
    const long long nrows = npairs * sdp::VT * sdp::BM;
    const float2* xv = static_cast<const float2*>(x);
    sdp::dm_prep_voxels<<<(unsigned)((nrows + 255) / 256), 256, 0, st>>>(xv, nvox, dm->K, dm->KS, nrows, dm->xh);
    GemmArgs a{dm->xh, dm->bh, nvox, (int)npairs, dm->ntiles, dm->best_score, dm->best, dm->status,
               dm->timeout_ns, dm->withhold_tile};
    const unsigned grid = (unsigned)std::min<long long>(npairs, dm->nsm);
    const int smem = std::max(dm->KS == 1 ? sdp::score_smem_bytes<1>() : sdp::score_smem_bytes<2>(), sdp::kMinSmem);
    if (dm->KS == 1)
        sdp::dm_score_kernel<1><<<grid, sdp::kThreadsG, smem, st>>>(a);
    else
        sdp::dm_score_kernel<2><<<grid, sdp::kThreadsG, smem, st>>>(a);
    sdp::dm_refine<<<(unsigned)((nvox + 8 * sdp::RV - 1) / (8 * sdp::RV)), 256, 0, st>>>(xv, nvox, dm->K, dm->best_score, dm->best, dm->dhat,
                                                               dm->inv_norm,
                                                               dm->P, 2 * dm->ntiles, dm->params, idx,
                                                               static_cast<float2*>(pd),
                                                               reinterpret_cast<float2*>(qmap));
    sdp::note_launches(3);
    if (cudaGetLastError() != cudaSuccess) return SDP_ERR_CUDA;
    return SDP_OK;
}

int sdp_dm_set_wait_test(sdp_dm_t dm, int32_t withhold_tile, int64_t timeout_ns) {
    if (!dm || withhold_tile < -1 || withhold_tile >= dm->ntiles) return SDP_ERR_INVALID_ARG;
    if (timeout_ns != 0 && (timeout_ns < 1000 || timeout_ns > 10000000000LL)) return SDP_ERR_INVALID_ARG;
    dm->withhold_tile = withhold_tile;
    dm->timeout_ns = timeout_ns == 0 ? sdp::kTimeoutNs : (unsigned long long)timeout_ns;
    return SDP_OK;
}

int sdp_dm_status(sdp_dm_t dm, void* stream) {
    if (!dm) return SDP_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int h = 0;
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaMemcpy(&h, dm->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemset(dm->status, 0, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return SDP_ERR_CUDA;
    }
    return h;
}

int sdp_dm_info(sdp_dm_t dm, int64_t* out, int32_t cap) {
    if (!dm || !out || cap < 0) return SDP_ERR_INVALID_ARG;
    const int64_t v[8] = {dm->P,
                          dm->K,
                          dm->KS,
                          dm->ntiles,
                          dm->max_vox,
                          (int64_t)dm->bytes,
                          (int64_t)std::min<long long>(pairs_for(dm->max_vox), dm->nsm),
                          (int64_t)dm->ntiles * 2 * sdp::BN * 16 * dm->KS};
    for (int i = 0; i < cap && i < 8; ++i) out[i] = v[i];
    return SDP_OK;
}

}  // extern "C"
