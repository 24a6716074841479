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
// for one channel and a segment of SEG planes; in the value kernel warp w of
// the block holds row i2 = y0 + w (in the gradient kernel rows y0 + 2w and
// y0 + 2w + 1), lane l holds i3 = x0 + l, and every thread walks its column
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

// Gradient kernel: a thread owns two rows of its column, A = y0 + 2w and
// B = A + 1 (warp w of 4; the block still covers a TX x TY tile).  Row B's
// "point above" is row A, so q_2 of the point above B is row A's own q_2, and
// x(p, B) is row A's axis-2 neighbour: per plane the pair needs x(p+1, A),
// x(p+1, B), x(p, B+1) and x(p+1, A-1) (in the last lane also x(p, A, i3+1),
// x(p, B, i3+1), x(p, A-1, i3+1); in lane 0 x(p+1, A, i3-1), x(p+1, B, i3-1),
// x(p, B+1, i3-1)).
constexpr int kThreadsG = TX * TY / 2;
constexpr int PFG = 3;             // planes of loads in flight per thread (10 values per plane)

struct Offs2 {
    int a, b, bd, au;              // rows A, B, B + 1, A - 1 at column i3
    int rta, rtb, urt;             // column i3 + 1 of rows A, B, A - 1
    int lfa, lfb, lfbd;            // column i3 - 1 of rows A, B, B + 1
    bool up_a, dn_a, dn_b, rt, lf; // the neighbour lies on the volume
};

__device__ __forceinline__ Offs2 offsets2_of(const Vol& v, int ia, int i3) {
    Offs2 o;
    auto row = [&](int r) { return min(max(r, 0), v.N2 - 1) * v.N3; };
    const int c0 = min(i3, v.N3 - 1);
    const int crt = min(c0 + 1, v.N3 - 1), clf = max(c0 - 1, 0);
    const int ra = row(ia), rb = row(ia + 1), rbd = row(ia + 2), rau = row(ia - 1);
    o.a = ra + c0;
    o.b = rb + c0;
    o.bd = rbd + c0;
    o.au = rau + c0;
    o.rta = ra + crt;
    o.rtb = rb + crt;
    o.urt = rau + crt;
    o.lfa = ra + clf;
    o.lfb = rb + clf;
    o.lfbd = rbd + clf;
    o.up_a = ia > 0;
    o.dn_a = ia + 1 < v.N2;
    o.dn_b = ia + 2 < v.N2;
    o.rt = i3 + 1 < v.N3;
    o.lf = i3 > 0;
    return o;
}

struct StepG2 {
    float2 ba, bb, dnb, ub;        // x(p+1, A), x(p+1, B), x(p, B+1), x(p+1, A-1)
    float2 rta, rtb, urt;          // last lane
    float2 lfba, lfbb, lfdb;       // lane 0
};

__device__ __forceinline__ StepG2 load_g2(const float2* __restrict__ xk, const Vol& v, const Offs2& o, int p,
                                          bool first_lane, bool last_lane) {
    const int pc = min(p, v.N1 - 1) * (int)v.plane, pn = min(p + 1, v.N1 - 1) * (int)v.plane;
    const float2 z = make_float2(0.f, 0.f);
    StepG2 r;
    r.ba = ldx(xk + pn + o.a);
    r.bb = ldx(xk + pn + o.b);
    r.dnb = ldx(xk + pc + o.bd);
    r.ub = ldx(xk + pn + o.au);
    r.rta = last_lane ? ldx(xk + pc + o.rta) : z;
    r.rtb = last_lane ? ldx(xk + pc + o.rtb) : z;
    r.urt = last_lane ? ldx(xk + pc + o.urt) : z;
    r.lfba = first_lane ? ldx(xk + pn + o.lfa) : z;
    r.lfbb = first_lane ? ldx(xk + pn + o.lfb) : z;
    r.lfdb = first_lane ? ldx(xk + pc + o.lfbd) : z;
    return r;
}

// q = D x / s at one point from its three forward differences.
__device__ __forceinline__ void qvec(float2 d1, float2 d2, float2 d3, float eps2, float2& q1, float2& q2, float2& q3) {
    const float is = rsqrtf(smag2(d1, d2, d3, eps2));              // 1 / s (hardware rsqrt)
    q1 = scl(d1, is);
    q2 = scl(d2, is);
    q3 = scl(d3, is);
}

// gradient: out = (accumulate ? out : 0) + lambda * (*scale) * grad TV.  q_1 of
// the plane before is the register kept from the previous step (a warm-up step
// at pb - 1 supplies it); q_3 of the point to the left comes from the lane to
// the left (lane 0 forms it from the column left of the tile); q_2 of the point
// above row A is formed from row A - 1's values, that of row B is row A's.
__global__ void __launch_bounds__(kThreadsG, 4) tv_grad_kernel(const float2* __restrict__ x, Vol v, float eps,
                                                              float lambda, const float* __restrict__ scale,
                                                              float2* __restrict__ out, int accumulate) {
    int bi = blockIdx.x;
    const int t3 = bi % v.nt3;
    bi /= v.nt3;
    const int t2 = bi % v.nt2;
    const int sg = bi / v.nt2;
    const int lane = threadIdx.x & 31;
    const int i3 = t3 * TX + lane;
    const int ia = t2 * TY + 2 * (threadIdx.x >> 5);
    const int pb = sg * SEG, pe = min(v.N1, pb + SEG);
    const bool in_a = ia < v.N2 && i3 < v.N3, in_b = ia + 1 < v.N2 && i3 < v.N3;
    const Offs2 o = offsets2_of(v, ia, i3);
    const float eps2 = eps * eps;
    const float f = lambda * (scale ? __ldg(scale) : 1.f);
    const float2 z = make_float2(0.f, 0.f);
    const float2* xk = x + (long long)blockIdx.y * v.nvox;
    float2* ok = out + (long long)blockIdx.y * v.nvox;
    const int plane = (int)v.plane;
    const bool first_lane = lane == 0, last_lane = lane == 31;
    const int p0 = pb > 0 ? pb - 1 : 0;
    float2 xa = ldx(xk + p0 * plane + o.a);                          // x(p, A)
    float2 xb = ldx(xk + p0 * plane + o.b);                          // x(p, B)
    float2 up = ldx(xk + p0 * plane + o.au);                         // x(p, A - 1)
    float2 lfa = first_lane ? ldx(xk + p0 * plane + o.lfa) : z;      // x(p, A, i3 - 1), lane 0
    float2 lfb = first_lane ? ldx(xk + p0 * plane + o.lfb) : z;      // x(p, B, i3 - 1), lane 0
    StepG2 q[PFG];
#pragma unroll
    for (int j = 0; j < PFG; ++j) q[j] = load_g2(xk, v, o, p0 + j, first_lane, last_lane);
    float2 q1pa = z, q1pb = z;                                       // q_1 of the plane before
#pragma unroll
    for (int j = 0; j <= SEG; ++j) {
        const int p = p0 + j;
        StepG2 cur = q[j % PFG];
        if (j + PFG <= SEG) q[j % PFG] = load_g2(xk, v, o, p + PFG, first_lane, last_lane);
        const float2 sra = shfl_down1(xa), srb = shfl_down1(xb), sru = shfl_down1(up);
        if (!last_lane) {
            cur.rta = sra;
            cur.rtb = srb;
            cur.urt = sru;
        }
        if (p + 1 >= v.N1) {                                         // no plane after: D1 = 0
            cur.ba = xa;
            cur.bb = xb;
            cur.ub = up;
            cur.lfba = lfa;
            cur.lfbb = lfb;
        }
        if (!o.rt) {
            cur.rta = xa;
            cur.rtb = xb;
            cur.urt = up;
        }
        const float2 dna = o.dn_a ? xb : xa;                          // x(p, A+1) or no difference
        const float2 lfda = o.dn_a ? lfb : lfa;
        if (!o.dn_b) {
            cur.dnb = xb;
            cur.lfdb = lfb;
        }
        float2 q1a, q2a, q3a, q1b, q2b, q3b;
        qvec(sub(cur.ba, xa), sub(dna, xa), sub(cur.rta, xa), eps2, q1a, q2a, q3a);
        qvec(sub(cur.bb, xb), sub(cur.dnb, xb), sub(cur.rtb, xb), eps2, q1b, q2b, q3b);
        // q_2 of the point above row A (0 off the volume)
        const float2 e2 = sub(xa, up);
        float2 q2ua = scl(e2, rsqrtf(smag2(sub(cur.ub, up), e2, sub(cur.urt, up), eps2)));
        if (!o.up_a) q2ua = z;
        // q_3 of the points to the left (0 off the volume)
        float2 q3la = shfl_up1(q3a), q3lb = shfl_up1(q3b);
        if (first_lane) {
            const float2 ga = sub(xa, lfa), gb = sub(xb, lfb);
            q3la = scl(ga, rsqrtf(smag2(sub(cur.lfba, lfa), sub(lfda, lfa), ga, eps2)));
            q3lb = scl(gb, rsqrtf(smag2(sub(cur.lfbb, lfb), sub(cur.lfdb, lfb), gb, eps2)));
        }
        if (!o.lf) {
            q3la = z;
            q3lb = z;
        }
        if (p >= pb && p < pe) {
            float2* dst = ok + p * plane + o.a;
            if (in_a) {
                float2 g = make_float2(f * (q1pa.x - q1a.x + q2ua.x - q2a.x + q3la.x - q3a.x),
                                       f * (q1pa.y - q1a.y + q2ua.y - q2a.y + q3la.y - q3a.y));
                if (accumulate) {
                    const float2 prev = *dst;
                    g.x += prev.x;
                    g.y += prev.y;
                }
                *dst = g;
            }
            if (in_b) {
                float2* dstb = dst + v.N3;
                float2 g = make_float2(f * (q1pb.x - q1b.x + q2a.x - q2b.x + q3lb.x - q3b.x),
                                       f * (q1pb.y - q1b.y + q2a.y - q2b.y + q3lb.y - q3b.y));
                if (accumulate) {
                    const float2 prev = *dstb;
                    g.x += prev.x;
                    g.y += prev.y;
                }
                *dstb = g;
            }
        }
        q1pa = q1a;
        q1pb = q1b;
        xa = cur.ba;
        xb = cur.bb;
        up = cur.ub;
        lfa = cur.lfba;
        lfb = cur.lfbb;
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
    tv_grad_kernel<<<grid, kThreadsG, 0, st>>>(x, v, eps, lambda, scale, out, accumulate);
    return cudaGetLastError();
}

}  // namespace sdp
