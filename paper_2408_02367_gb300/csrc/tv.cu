// Spatial total-variation penalty of StoDIP (Sec. 2.1, Algorithm 1 line 6:
// loss = L_c + lambda TV(x_hat)).  The paper does not define TV; the reading
// implemented is the isotropic, epsilon-smoothed TV of every subspace channel,
// forward differences with a zero difference at the last index of each axis:
//
//   s_k(n)  = sqrt(|D1 x_k(n)|^2 + |D2 x_k(n)|^2 + |D3 x_k(n)|^2 + eps^2)
//   TV(x)   = sum_k sum_n s_k(n),      D_d x(n) = x(n + e_d) - x(n)  (0 at n_d = N_d - 1)
//   grad(m) = sum_d [ q_d(m - e_d) - q_d(m) ],   q_d = D_d x / s  (q_d = 0 off the volume)
//
// grad is dTV/dRe + i dTV/dIm (PyTorch's convention).
//
// Both kernels march along axis 1.  A block owns a TY x TX tile of (i2, i3)
// for one channel and a segment of SEG planes; warp w of the block holds row
// i2 = y0 + w, lane l holds i3 = x0 + l, and every thread walks its column
// (i2, i3) plane by plane.  The axis-3 neighbours come from warp shuffles
// (the last lane loads the one past the tile), the axis-2 neighbours are
// loads of the neighbouring rows (hits in L1 or L2: those rows are another
// warp's own column), and the axis-1 neighbour of plane p is the column's
// value of plane p + 1, which is carried to the next plane in a register.
// Every load address is clamped onto the volume and the boundary cases are
// selects, and the loads of the next PF steps are kept in flight in
// registers (a ring indexed at compile time in the fully unrolled plane loop),
// so each warp has several planes of loads outstanding; each x value comes
// from DRAM about once per launch, and no barrier or shared-memory staging
// sits in the loop.
//
// The value is reduced in a fixed order (bitwise repeatable): float32 within
// a thread (at most SEG terms) and a warp, float64 across the warps of a
// block and across blocks (the last block to finish adds the block partials
// in index order).
#include "sdp_internal.cuh"

namespace sdp {
namespace {

constexpr int TX = 32;             // tile along i3 (the lanes of a warp)
constexpr int TY = 8;              // tile along i2 (the warps of a block)
constexpr int SEG = 16;            // planes along i1 per block
constexpr int kThreads = TX * TY;
constexpr unsigned kFull = 0xffffffffu;

struct Vol {
    int N1, N2, N3;
    int nt3, nt2, nseg;            // tiles along i3, i2 and segments along i1
    long long plane;               // N2 * N3
    long long nvox;
};

struct Col {
    int k, i2, i3, pb, pe;         // channel, column, planes [pb, pe)
    int lane, x0;
    bool inside;                   // (i2, i3) on the volume
};

__device__ __forceinline__ Col column_of(const Vol& v) {
    Col c;
    int b = blockIdx.x;
    const int t3 = b % v.nt3;
    b /= v.nt3;
    const int t2 = b % v.nt2;
    const int sg = b / v.nt2;
    c.k = blockIdx.y;
    c.lane = threadIdx.x & 31;
    c.x0 = t3 * TX;
    c.i3 = c.x0 + c.lane;
    c.i2 = t2 * TY + (threadIdx.x >> 5);
    c.pb = sg * SEG;
    c.pe = min(v.N1, c.pb + SEG);
    c.inside = c.i2 < v.N2 && c.i3 < v.N3;
    return c;
}

__device__ __forceinline__ float2 ldx(const float2* __restrict__ p) { return __ldg(p); }
__device__ __forceinline__ float2 sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 scl(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 shfl_down1(float2 a) {
    return make_float2(__shfl_down_sync(kFull, a.x, 1), __shfl_down_sync(kFull, a.y, 1));
}
__device__ __forceinline__ float2 shfl_up1(float2 a) {
    return make_float2(__shfl_up_sync(kFull, a.x, 1), __shfl_up_sync(kFull, a.y, 1));
}
__device__ __forceinline__ float smag2(float2 d1, float2 d2, float2 d3, float eps2) {
    return d1.x * d1.x + d1.y * d1.y + d2.x * d2.x + d2.y * d2.y + d3.x * d3.x + d3.y * d3.y + eps2;
}

// Fixed-order block reduction: float32 warp butterflies, then the warps in order in float64.
__device__ __forceinline__ double block_sum_f(float v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kThreads / 32; ++w) s += red[w];
    return s;
}

__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kThreads / 32; ++w) s += red[w];
    return s;
}

// One block partial into partials[blockIdx]; the last block to arrive writes
// lambda * (the fixed-order sum of all partials) to *out and rearms the counter.
__device__ __forceinline__ void finish_value(double bs, float lambda, double* __restrict__ partials,
                                             unsigned int* __restrict__ counter, float* __restrict__ out,
                                             double* red) {
    __shared__ bool s_last;
    const unsigned nblk = gridDim.x * gridDim.y;
    if (threadIdx.x == 0) {
        partials[(long long)blockIdx.y * gridDim.x + blockIdx.x] = bs;
        __threadfence();
        s_last = (atomicAdd(counter, 1u) == nblk - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double tot = 0.0;
    for (unsigned i = threadIdx.x; i < nblk; i += kThreads) tot += __ldcg(partials + i);
    __syncthreads();                              // red is reused
    tot = block_sum(tot, red);
    if (threadIdx.x == 0) {
        *out = (float)((double)lambda * tot);
        *counter = 0u;
    }
}

// Offsets within one channel of the column and of its neighbours, clamped onto
// the volume so that every load of the plane loop is valid and unconditional
// (a clamped neighbour is never used: the difference it would feed is zero).
struct Offs {
    int o0, dn, up, rt, urt, lf, dnlf;
    bool has_dn, has_up, has_rt, has_lf;
};

__device__ __forceinline__ Offs offsets_of(const Vol& v, const Col& c) {
    Offs o;
    const int i2 = min(c.i2, v.N2 - 1), i3 = min(c.i3, v.N3 - 1);
    o.has_dn = c.i2 + 1 < v.N2;
    o.has_up = c.i2 > 0;
    o.has_rt = c.i3 + 1 < v.N3;
    o.has_lf = c.i3 > 0;
    const int r_dn = (i2 + 1 < v.N2 ? i2 + 1 : i2) * v.N3, r_up = (i2 > 0 ? i2 - 1 : i2) * v.N3, r0 = i2 * v.N3;
    const int c_rt = i3 + 1 < v.N3 ? i3 + 1 : i3, c_lf = i3 > 0 ? i3 - 1 : i3;
    o.o0 = r0 + i3;
    o.dn = r_dn + i3;
    o.up = r_up + i3;
    o.rt = r0 + c_rt;
    o.urt = r_up + c_rt;
    o.lf = r0 + c_lf;
    o.dnlf = r_dn + c_lf;
    return o;
}

constexpr int PF = 4;              // planes of loads kept in flight per thread

// The loads of one step of the value kernel: x(p+1, i2, i3), x(p, i2+1, i3)
// and, in the last lane, x(p, i2, i3+1).
struct StepV {
    float2 b, dn, rt;
};

__device__ __forceinline__ StepV load_v(const float2* __restrict__ xk, const Vol& v, const Offs& o, int p,
                                        bool last_lane) {
    const int pc = min(p, v.N1 - 1), pn = min(p + 1, v.N1 - 1);
    StepV r;
    r.b = ldx(xk + pn * (int)v.plane + o.o0);
    r.dn = ldx(xk + pc * (int)v.plane + o.dn);
    r.rt = last_lane ? ldx(xk + pc * (int)v.plane + o.rt) : make_float2(0.f, 0.f);
    return r;
}

// value: lambda * TV(x)
__global__ void __launch_bounds__(kThreads, 4) tv_value_kernel(const float2* __restrict__ x, Vol v, float eps,
                                                              float lambda, double* __restrict__ partials,
                                                              unsigned int* __restrict__ counter,
                                                              float* __restrict__ out) {
    __shared__ double red[kThreads / 32];
    const Col c = column_of(v);
    const Offs o = offsets_of(v, c);
    const float eps2 = eps * eps;
    const float2* xk = x + (long long)c.k * v.nvox;
    const bool last_lane = c.lane == 31;
    float2 a = ldx(xk + c.pb * (int)v.plane + o.o0);               // x(p, i2, i3)
    StepV q[PF];
#pragma unroll
    for (int j = 0; j < PF; ++j) q[j] = load_v(xk, v, o, c.pb + j, last_lane);
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < SEG; ++j) {
        const int p = c.pb + j;
        StepV cur = q[j % PF];
        if (j + PF < SEG) q[j % PF] = load_v(xk, v, o, p + PF, last_lane);
        const float2 sh = shfl_down1(a);
        if (!last_lane) cur.rt = sh;
        if (p + 1 >= v.N1) cur.b = a;
        if (!o.has_dn) cur.dn = a;
        if (!o.has_rt) cur.rt = a;
        const float s2 = smag2(sub(cur.b, a), sub(cur.dn, a), sub(cur.rt, a), eps2);
        if (c.inside && p < c.pe) acc += s2 * rsqrtf(s2);            // s = s2 / sqrt(s2), s2 >= eps^2 > 0
        a = cur.b;
    }
    finish_value(block_sum_f(acc, red), lambda, partials, counter, out, red);
}

// The loads of one step of the gradient kernel: x(p+1, i2, i3), x(p, i2+1, i3),
// x(p+1, i2-1, i3); in the last lane x(p, i2, i3+1) and x(p, i2-1, i3+1); in
// lane 0 x(p+1, i2, i3-1) and x(p, i2+1, i3-1).
struct StepG {
    float2 b, dn, ub, rt, urt, lfb, lfd;
};

__device__ __forceinline__ StepG load_g(const float2* __restrict__ xk, const Vol& v, const Offs& o, int p,
                                        bool first_lane, bool last_lane) {
    const int pc = min(p, v.N1 - 1) * (int)v.plane, pn = min(p + 1, v.N1 - 1) * (int)v.plane;
    const float2 z = make_float2(0.f, 0.f);
    StepG r;
    r.b = ldx(xk + pn + o.o0);
    r.dn = ldx(xk + pc + o.dn);
    r.ub = ldx(xk + pn + o.up);
    r.rt = last_lane ? ldx(xk + pc + o.rt) : z;
    r.urt = last_lane ? ldx(xk + pc + o.urt) : z;
    r.lfb = first_lane ? ldx(xk + pn + o.lf) : z;
    r.lfd = first_lane ? ldx(xk + pc + o.dnlf) : z;
    return r;
}

// gradient: out = (accumulate ? out : 0) + lambda * (*scale) * grad TV.  Besides
// its own q_d, a thread forms q_2 of the point above it (i2 - 1) from that
// row's values, and takes q_3 of the point left of it (i3 - 1) from the lane
// to its left (lane 0 forms it from the column left of the tile); q_1 of the
// plane before is the register kept from the previous step (a warm-up step at
// pb - 1 supplies it).
__global__ void __launch_bounds__(kThreads, 2) tv_grad_kernel(const float2* __restrict__ x, Vol v, float eps,
                                                             float lambda, const float* __restrict__ scale,
                                                             float2* __restrict__ out, int accumulate) {
    const Col c = column_of(v);
    const Offs o = offsets_of(v, c);
    const float eps2 = eps * eps;
    const float f = lambda * (scale ? __ldg(scale) : 1.f);
    const float2 z = make_float2(0.f, 0.f);
    const float2* xk = x + (long long)c.k * v.nvox;
    float2* ok = out + (long long)c.k * v.nvox;
    const int plane = (int)v.plane;
    const bool first_lane = c.lane == 0, last_lane = c.lane == 31;
    const int p0 = c.pb > 0 ? c.pb - 1 : 0;
    float2 a = ldx(xk + p0 * plane + o.o0);                          // x(p, i2, i3)
    float2 up = ldx(xk + p0 * plane + o.up);                         // x(p, i2 - 1, i3)
    float2 lf = first_lane ? ldx(xk + p0 * plane + o.lf) : z;        // x(p, i2, i3 - 1), lane 0
    StepG q[PF];
#pragma unroll
    for (int j = 0; j < PF; ++j) q[j] = load_g(xk, v, o, p0 + j, first_lane, last_lane);
    float2 q1p = z;                                                  // q_1(p - 1, i2, i3)
#pragma unroll
    for (int j = 0; j <= SEG; ++j) {
        const int p = p0 + j;
        StepG cur = q[j % PF];
        if (j + PF <= SEG) q[j % PF] = load_g(xk, v, o, p + PF, first_lane, last_lane);
        const float2 sr = shfl_down1(a), sur = shfl_down1(up);
        if (!last_lane) {
            cur.rt = sr;
            cur.urt = sur;
        }
        if (p + 1 >= v.N1) {
            cur.b = a;
            cur.ub = up;
            cur.lfb = lf;
        }
        if (!o.has_dn) {
            cur.dn = a;
            cur.lfd = lf;
        }
        if (!o.has_rt) {
            cur.rt = a;
            cur.urt = up;
        }
        const float2 d1 = sub(cur.b, a), d2 = sub(cur.dn, a), d3 = sub(cur.rt, a);
        const float is = rsqrtf(smag2(d1, d2, d3, eps2));           // 1 / s (hardware rsqrt)
        const float2 q1 = scl(d1, is), q2 = scl(d2, is), q3 = scl(d3, is);
        const float2 e2 = sub(a, up);                                // q_2(p, i2 - 1, i3)
        float2 q2u = scl(e2, rsqrtf(smag2(sub(cur.ub, up), e2, sub(cur.urt, up), eps2)));
        if (!o.has_up) q2u = z;
        float2 q3l = shfl_up1(q3);                                   // q_3(p, i2, i3 - 1)
        if (first_lane) {
            const float2 g3 = sub(a, lf);
            q3l = scl(g3, rsqrtf(smag2(sub(cur.lfb, lf), sub(cur.lfd, lf), g3, eps2)));
        }
        if (!o.has_lf) q3l = z;
        if (c.inside && p >= c.pb && p < c.pe) {
            float2 g = make_float2(f * (q1p.x - q1.x + q2u.x - q2.x + q3l.x - q3.x),
                                   f * (q1p.y - q1.y + q2u.y - q2.y + q3l.y - q3.y));
            float2* dst = ok + p * plane + o.o0;
            if (accumulate) {
                const float2 prev = *dst;
                g.x += prev.x;
                g.y += prev.y;
            }
            *dst = g;
        }
        q1p = q1;
        a = cur.b;
        up = cur.ub;
        lf = cur.lfb;
    }
}

Vol make_vol(const Geo& g) {
    Vol v;
    v.N1 = g.N[0];
    v.N2 = g.N[1];
    v.N3 = g.N[2];
    v.nt3 = (v.N3 + TX - 1) / TX;
    v.nt2 = (v.N2 + TY - 1) / TY;
    v.nseg = (v.N1 + SEG - 1) / SEG;
    v.plane = (long long)v.N2 * v.N3;
    v.nvox = v.plane * v.N1;
    return v;
}

}  // namespace

long long tv_partials(int K, int N1, int N2, int N3) {
    return (long long)K * ((N3 + TX - 1) / TX) * ((N2 + TY - 1) / TY) * ((N1 + SEG - 1) / SEG);
}

cudaError_t launch_tv_value(const Geo& g, const float2* x, float eps, float lambda, double* partials,
                            unsigned int* counter, float* out, cudaStream_t st) {
    const Vol v = make_vol(g);
    if (v.nvox >= (1LL << 31)) return cudaErrorInvalidValue;         // offsets within a channel are 32-bit
    const dim3 grid((unsigned)(v.nt3 * v.nt2 * v.nseg), (unsigned)g.K);
    tv_value_kernel<<<grid, kThreads, 0, st>>>(x, v, eps, lambda, partials, counter, out);
    return cudaGetLastError();
}

cudaError_t launch_tv_grad(const Geo& g, const float2* x, float eps, float lambda, const float* scale, float2* out,
                           int accumulate, cudaStream_t st) {
    const Vol v = make_vol(g);
    if (v.nvox >= (1LL << 31)) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)(v.nt3 * v.nt2 * v.nseg), (unsigned)g.K);
    tv_grad_kernel<<<grid, kThreads, 0, st>>>(x, v, eps, lambda, scale, out, accumulate);
    return cudaGetLastError();
}

}  // namespace sdp
