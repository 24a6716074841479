// C ABI of the subspace multicoil NUFFT operator (declared in include/stodip_op.h):
// plan construction on the host (grid sizes, Kaiser-Bessel beta and
// deapodisation, FFT factorisation and twiddles, grid coordinates, bin sort,
// spread incidence lists), and the launch sequences of the forward operator
// A_c and its adjoint (StoDIP Sec. 2 Eq. 1, Sec. 2.1 Eq. 3, Algorithm 1).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "batch.cuh"
#include "sdp_internal.cuh"

using namespace sdp;

namespace {

constexpr double kPi = 3.14159265358979323846;
std::atomic<long long> g_launches{0};

struct ProfRec {
    int stage;
    cudaEvent_t a, b;
};

}  // namespace

void sdp::note_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

struct sdp_plan_s {
    int dev = 0;
    Geo geo{};
    int64_t n[3] = {0, 0, 0};
    int64_t M[3] = {0, 0, 0};
    double sigma = 0, beta = 0;
    int maxB = 0;
    uint32_t flags = 0;
    FftAxis ax[3]{};
    int bs[3] = {0, 0, 0};
    int nb[3] = {0, 0, 0};
    int spread_chunk = 0;
    int interp_threads = 0;   // resolved CTA size of the interpolation kernel
    int spread_coils = 0;     // coils per spread warp: 0 = two where they fit, 1 = one
    int interp_run = 1;       // consecutive samples per interpolation warp run
    int interp_coils = 0;     // coils per interpolation sweep over the samples: 0 = all
    int interp_tiled = 0;     // 1: the tiled interpolation where it has a kernel (interp_tiles.cu)
    int nt[3] = {0, 0, 0};    // interpolation tiles per axis
    int n_itiles = 0;         // tiled interpolation work items
    int wait_test_row = -1;   // test hook (sdp_plan_set_wait_test): a tile row the first CTA withholds
    long long wait_test_ns = 0;   // and the limit of the tiled kernel's waits (0: one second)
    int nbins = 0;
    int nsub = 0;
    long long ninc = 0;
    long long slots_per_b = 0;
    // device memory
    float4* pts = nullptr;
    int* tframe = nullptr;
    float* wts = nullptr;    // [J][3W] Kaiser-Bessel weights of the sorted samples
    float2* V = nullptr;
    float2* S = nullptr;
    float* dinv = nullptr;   // [N1 | N2 | N3]
    float2* tw = nullptr;    // [M1 | M2 | M3]
    int* inc = nullptr;
    SubProb* subs = nullptr;
    int4* itiles = nullptr;  // tiled interpolation work items (flat tile index, first sample, count, 0), heaviest first
    float2* partials = nullptr;
    int* counters = nullptr;
    int* status = nullptr;
    double* loss_partials = nullptr;
    unsigned int* loss_counter = nullptr;
    double* tv_part = nullptr;
    unsigned int* tv_counter = nullptr;
    // Grid workspaces, channel-interleaved: a call with nk channels holds
    // [b][i1][i2][i3][kk] (kk fastest), so the W x nk values one row of a
    // Kaiser-Bessel window touches along axis 3 are one contiguous run.
    float2* bufA = nullptr;
    float2* bufB = nullptr;
    size_t workspace_bytes = 0;
    size_t total_bytes = 0;
    std::vector<void*> allocs;
    // profiling
    bool prof = false;
    std::vector<ProfRec> prof_used;
    std::vector<ProfRec> prof_free;
    double prof_ms[kNumStages] = {0};
    long long prof_n[kNumStages] = {0};
};

namespace {

bool smooth235(long long m) {
    for (int p : {2, 3, 5})
        while (m % p == 0) m /= p;
    return m == 1;
}

long long grid_len(long long n, double sigma, int W) {
    long long m = std::max((long long)std::ceil(sigma * (double)n), 2LL * W);
    while ((m % 2) || !smooth235(m)) ++m;
    return m;
}

double i0(double x) { return std::cyl_bessel_i(0.0, x); }

// Continuous Fourier transform of the normalised Kaiser-Bessel window.
double kb_ft(double xi, int W, double beta) {
    const double z2 = beta * beta - (kPi * W * xi) * (kPi * W * xi);
    const double z = std::sqrt(std::fabs(z2));
    double v;
    if (z == 0.0)
        v = 1.0;
    else if (z2 > 0)
        v = std::sinh(z) / z;
    else
        v = std::sin(z) / z;
    return W * v / i0(beta);
}

template <typename T>
int dev_alloc(sdp_plan_s* p, T** ptr, size_t count) {
    *ptr = nullptr;
    if (count == 0) count = 1;
    void* q = nullptr;
    if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return SDP_ERR_OOM;
    }
    p->allocs.push_back(q);
    p->total_bytes += count * sizeof(T);
    *ptr = static_cast<T*>(q);
    return SDP_OK;
}

void free_plan(sdp_plan_s* p) {
    if (!p) return;
    cudaDeviceSynchronize();
    for (void* q : p->allocs) cudaFree(q);
    for (auto& r : p->prof_used) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto& r : p->prof_free) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    delete p;
}

#define SDP_TRY(expr)                      \
    do {                                   \
        int _rc = (expr);                  \
        if (_rc != SDP_OK) return _rc;     \
    } while (0)

#define SDP_CUDA(expr)                     \
    do {                                   \
        if ((expr) != cudaSuccess) {       \
            cudaGetLastError();            \
            return SDP_ERR_CUDA;           \
        }                                  \
    } while (0)

// Grid coordinate of one axis, bit-for-bit the definition of the oracle:
// g = omega * (M / 2 pi) in float64, wrapped into [0, M), rounded to float32,
// a float32 equal to M becomes 0.  (Built with -ffp-contract=off.)
float grid_coord(float omega, long long M) {
    const double m = (double)M;
    const double s = m / (2.0 * kPi);
    double g = (double)omega * s;
    if (g < 0.0) g = g + m;
    if (g >= m) g = g - m;
    float g32 = (float)g;
    if (g32 >= (float)m) g32 = 0.0f;
    return g32;
}

int build_plan(sdp_plan_s* p, const sdp_plan_desc* d, const sdp_tuning* tn, cudaStream_t st) {
    const int W = d->width;
    const int K = d->K;
    const long long J = d->J;
    for (int a = 0; a < 3; ++a) {
        p->n[a] = d->n[a];
        p->M[a] = grid_len(d->n[a], d->oversamp, W);
        if (p->M[a] > (1 << 14)) return SDP_ERR_UNSUPPORTED;
    }
    const long long G = p->M[0] * p->M[1] * p->M[2];
    const long long nvox = p->n[0] * p->n[1] * p->n[2];
    // one coil's channel-interleaved grid [M1][M2][M3][K] is indexed with 32-bit offsets
    if (G * K >= (1LL << 31) || nvox >= (1LL << 31)) return SDP_ERR_UNSUPPORTED;
    p->sigma = d->oversamp;
    const double arg = (W / d->oversamp) * (W / d->oversamp) * (d->oversamp - 0.5) * (d->oversamp - 0.5) - 0.8;
    if (!(arg > 0)) return SDP_ERR_UNSUPPORTED;
    p->beta = kPi * std::sqrt(arg);
    p->maxB = d->max_batch;
    p->flags = d->flags;
    Geo& g = p->geo;
    for (int a = 0; a < 3; ++a) {
        g.N[a] = (int)p->n[a];
        g.M[a] = (int)p->M[a];
    }
    g.W = W;
    g.K = K;
    g.T = d->T;
    g.C = d->C;
    g.J = (int)J;
    g.beta = (float)p->beta;
    g.inv_i0_beta = (float)(1.0 / i0(p->beta));
    g.halfW = (float)(0.5 * W);
    for (int a = 0; a < 3; ++a) {
        if (!fft_factor(g.M[a], &p->ax[a])) return SDP_ERR_UNSUPPORTED;
        p->ax[a].generic = tn ? tn->fft_engine : 0;
        p->ax[a].lines = tn ? tn->fft_lines : 0;
        p->ax[a].cols = tn ? tn->fft_cols : 0;
        p->ax[a].staged = tn ? tn->fft_staged : 0;
    }
    // interpolation CTA size: the 1024-thread kernel is built for W <= 4 only
    const int ithreads = tn ? tn->interp_threads : 0;
    if (ithreads == 1024 && W > 4) return SDP_ERR_UNSUPPORTED;
    p->interp_threads = ithreads ? ithreads : 256;
    p->spread_coils = tn ? tn->spread_coils : 0;
    p->interp_run = (tn && tn->interp_run) ? tn->interp_run : 1;
    p->interp_coils = tn ? tn->interp_coils : 0;
    p->interp_tiled = tn ? tn->interp_tiled : 0;

    // ---- host tables ----
    std::vector<float> dinv(p->n[0] + p->n[1] + p->n[2]);
    {
        size_t o = 0;
        for (int a = 0; a < 3; ++a)
            for (long long i = 0; i < p->n[a]; ++i) {
                const double nc = (double)(i - p->n[a] / 2);
                dinv[o++] = (float)(1.0 / kb_ft(nc / (double)p->M[a], W, p->beta));
            }
    }
    std::vector<float2> tw;
    for (int a = 0; a < 3; ++a) {
        std::vector<float2> t = fft_twiddles(g.M[a]);
        tw.insert(tw.end(), t.begin(), t.end());
    }

    // ---- trajectory -> grid coordinates, frames ----
    std::vector<float> traj((size_t)J * 3);
    SDP_CUDA(cudaMemcpyAsync(traj.data(), d->traj, traj.size() * sizeof(float), cudaMemcpyDeviceToHost, st));
    SDP_CUDA(cudaStreamSynchronize(st));
    std::vector<int> frame((size_t)J);
    for (int t = 0; t < d->T; ++t)
        for (long long j = d->frame_offsets[t]; j < d->frame_offsets[t + 1]; ++j) frame[j] = t;
    std::vector<float> gc((size_t)J * 3);
    for (long long j = 0; j < J; ++j) {
        const float* om = &traj[(size_t)j * 3];
        if (!(std::fabs(om[0]) <= (float)kPi + 1e-6f && std::fabs(om[1]) <= (float)kPi + 1e-6f &&
              std::fabs(om[2]) <= (float)kPi + 1e-6f))
            return SDP_ERR_INVALID_ARG;
        for (int a = 0; a < 3; ++a) gc[(size_t)j * 3 + a] = grid_coord(om[a], p->M[a]);
    }

    // ---- bins: B1 x 4 x B3 grid points, 8 x 4 x 8 unless tuned (one warp of the
    // spread; lanes own the B1 x 4 axis-3 columns, held in registers) ----
    int bs[3] = {8, 4, 8};
    if (tn)
        for (int a = 0; a < 3; ++a) bs[a] = tn->spread_bins[a];
    for (int a = 0; a < 3; ++a) {
        p->bs[a] = bs[a];
        p->nb[a] = (int)((p->M[a] + bs[a] - 1) / bs[a]);
    }
    const long long nbins = (long long)p->nb[0] * p->nb[1] * p->nb[2];
    if (nbins >= (1LL << 31)) return SDP_ERR_UNSUPPORTED;
    p->nbins = (int)nbins;

    // window start of each sample, and its sort key: samples are ordered by interpolation
    // tile (tiles of kTile^3 grid points: the tiled interpolation takes a tile's samples as
    // one range), then by spread bin within the tile (bins nest in tiles: kTile is a
    // multiple of every bin edge), both of the sample's own coordinate
    const float halfW = (float)(0.5 * W);
    const int kTile = interp_tile_edge();
    int bpt[3];
    for (int a = 0; a < 3; ++a) {
        bpt[a] = kTile / bs[a];
        p->nt[a] = (int)((p->M[a] + kTile - 1) / kTile);
    }
    const long long BPT = (long long)bpt[0] * bpt[1] * bpt[2];
    const long long ntiles = (long long)p->nt[0] * p->nt[1] * p->nt[2];
    const long long nkeys = ntiles * BPT;
    std::vector<int> m0((size_t)J * 3);
    std::vector<long long> skey((size_t)J);
    for (long long j = 0; j < J; ++j) {
        long long ti = 0, li = 0;
        for (int a = 0; a < 3; ++a) {
            const float gv = gc[(size_t)j * 3 + a];
            const float tt = gv - halfW;
            m0[(size_t)j * 3 + a] = (int)std::ceil(tt);
            int ba = (int)(gv / (float)bs[a]);
            if (ba >= p->nb[a]) ba = p->nb[a] - 1;
            ti = ti * p->nt[a] + ba / bpt[a];
            li = li * bpt[a] + ba % bpt[a];
        }
        skey[j] = ti * BPT + li;
    }
    // stable counting sort of samples by key
    std::vector<long long> cnt((size_t)nkeys + 1, 0);
    for (long long j = 0; j < J; ++j) cnt[(size_t)skey[j] + 1]++;
    for (long long b = 0; b < nkeys; ++b) cnt[(size_t)b + 1] += cnt[(size_t)b];
    std::vector<int> perm((size_t)J);   // sorted position -> original sample
    {
        std::vector<long long> cur(cnt.begin(), cnt.end() - 1);
        for (long long j = 0; j < J; ++j) perm[(size_t)cur[(size_t)skey[j]]++] = (int)j;
    }
    // the tiled interpolation's work items (flattened tile index, first sorted sample,
    // count), heaviest first: every non-empty tile, a dense one (the k-space centre holds
    // tiles of thousands of samples) cut into near-equal pieces of at most kTileItem
    // samples, each of which copies the tile's grid once per coil
    constexpr long long kTileItem = 512;
    std::vector<int4> itiles;
    for (long long t = 0; t < ntiles; ++t) {
        const long long c0 = cnt[(size_t)(t * BPT)], c1 = cnt[(size_t)((t + 1) * BPT)];
        const long long n = c1 - c0, parts = (n + kTileItem - 1) / kTileItem;
        for (long long q = 0; q < parts; ++q) {
            const long long a = c0 + n * q / parts, b = c0 + n * (q + 1) / parts;
            itiles.push_back(make_int4((int)t, (int)a, (int)(b - a), 0));
        }
    }
    std::stable_sort(itiles.begin(), itiles.end(), [](const int4& a, const int4& b) { return a.z > b.z; });
    p->n_itiles = (int)itiles.size();
    std::vector<float4> pts((size_t)J);
    std::vector<int> tf((size_t)J);
    for (long long s = 0; s < J; ++s) {
        const int j = perm[s];
        float4 q;
        q.x = gc[(size_t)j * 3 + 0];
        q.y = gc[(size_t)j * 3 + 1];
        q.z = gc[(size_t)j * 3 + 2];
        int jj = j;
        std::memcpy(&q.w, &jj, sizeof(int));
        pts[s] = q;
        tf[s] = frame[j];
    }

    // incidences: (bin, sorted sample) for every bin a window touches
    auto window_bins = [&](int m0a, int a, int* out) {
        int nbs = 0;
        for (int t = 0; t < W; ++t) {
            long long pos = m0a + t;
            if (pos < 0) pos += p->M[a];
            if (pos >= p->M[a]) pos -= p->M[a];
            const int b = (int)(pos / bs[a]);
            bool seen = false;
            for (int q = 0; q < nbs; ++q) seen |= (out[q] == b);
            if (!seen) out[nbs++] = b;
        }
        return nbs;
    };
    std::vector<long long> icnt(nbins + 1, 0);
    for (long long s = 0; s < J; ++s) {
        const int j = perm[s];
        int b1[kMaxWidth], b2[kMaxWidth], b3[kMaxWidth];
        const int n1 = window_bins(m0[(size_t)j * 3 + 0], 0, b1);
        const int n2 = window_bins(m0[(size_t)j * 3 + 1], 1, b2);
        const int n3 = window_bins(m0[(size_t)j * 3 + 2], 2, b3);
        for (int x = 0; x < n1; ++x)
            for (int y = 0; y < n2; ++y)
                for (int z = 0; z < n3; ++z)
                    icnt[((long long)b1[x] * p->nb[1] + b2[y]) * p->nb[2] + b3[z] + 1]++;
    }
    for (long long b = 0; b < nbins; ++b) icnt[b + 1] += icnt[b];
    const long long ninc = icnt[nbins];
    if (ninc >= (1LL << 31)) return SDP_ERR_UNSUPPORTED;
    p->ninc = ninc;
    std::vector<int> inc((size_t)std::max(ninc, 1LL));
    {
        std::vector<long long> cur(icnt.begin(), icnt.end() - 1);
        for (long long s = 0; s < J; ++s) {
            const int j = perm[s];
            int b1[kMaxWidth], b2[kMaxWidth], b3[kMaxWidth];
            const int n1 = window_bins(m0[(size_t)j * 3 + 0], 0, b1);
            const int n2 = window_bins(m0[(size_t)j * 3 + 1], 1, b2);
            const int n3 = window_bins(m0[(size_t)j * 3 + 2], 2, b3);
            for (int x = 0; x < n1; ++x)
                for (int y = 0; y < n2; ++y)
                    for (int z = 0; z < n3; ++z) {
                        const long long bin = ((long long)b1[x] * p->nb[1] + b2[y]) * p->nb[2] + b3[z];
                        inc[cur[bin]++] = (int)s;
                    }
        }
    }
    // each bin's incidences in order of axis-3 class (stable in sample order): the class
    // is o + W - 1 for the bin position o in [-(W-1), B3-1] of the window's first axis-3
    // tap, the same integer the spread kernel derives from the staged coordinate, which
    // runs each class with code for exactly the positions it covers.  Grids too short
    // along axis 3 for a window to meet a bin in one piece keep sample order.
    if (p->M[2] >= bs[2] + W - 1) {
        const int M3 = (int)p->M[2], ncls = bs[2] + W - 1;
        std::vector<int> tmp;
        std::vector<long long> ccnt((size_t)ncls + 2);
        for (long long b = 0; b < nbins; ++b) {
            const long long c0 = icnt[b], c1 = icnt[b + 1];
            if (c1 - c0 < 2) continue;
            const int lo3 = (int)(b % p->nb[2]) * bs[2];
            auto cls = [&](int s) {
                int d = lo3 - m0[(size_t)perm[s] * 3 + 2];
                d += d < 0 ? M3 : 0;
                d -= d >= M3 ? M3 : 0;
                const int c = (d < W ? -d : M3 - d) + W - 1;
                return (c >= 0 && c < ncls) ? c : ncls;
            };
            tmp.assign(inc.begin() + c0, inc.begin() + c1);
            std::fill(ccnt.begin(), ccnt.end(), 0);
            for (int s : tmp) ccnt[(size_t)cls(s) + 1]++;
            for (int c = 0; c <= ncls; ++c) ccnt[(size_t)c + 1] += ccnt[(size_t)c];
            for (int s : tmp) inc[(size_t)(c0 + ccnt[(size_t)cls(s)]++)] = s;
        }
    }
    // subproblems: every bin (empty ones too, they write zeros), chunks of at most kChunk
    long long kChunk = 512;
    if (tn)
        kChunk = tn->spread_chunk;
    else if (const char* ev = std::getenv("SDP_SPREAD_CHUNK"))
        kChunk = std::max(32LL, std::atoll(ev));
    p->spread_chunk = (int)kChunk;
    std::vector<SubProb> subs;
    long long slots = 0;
    for (long long b = 0; b < nbins; ++b) {
        const long long c0 = icnt[b], c1 = icnt[b + 1];
        const long long n = c1 - c0;
        const int nch = (int)std::max(1LL, (n + kChunk - 1) / kChunk);
        for (int ch = 0; ch < nch; ++ch) {
            SubProb sp;
            sp.bin = (int)b;
            sp.start = (int)(c0 + ch * kChunk);
            sp.count = (int)std::min(kChunk, n - ch * kChunk);
            if (sp.count < 0) sp.count = 0;
            sp.chunk = ch;
            sp.nchunks = nch;
            sp.slot = nch > 1 ? (int)slots : 0;
            subs.push_back(sp);
        }
        if (nch > 1) slots += nch;
    }
    // heaviest subproblems first
    std::stable_sort(subs.begin(), subs.end(), [](const SubProb& a, const SubProb& b) { return a.count > b.count; });
    p->nsub = (int)subs.size();
    p->slots_per_b = slots;

    // ---- device memory ----
    const size_t Kz = (size_t)K;
    SDP_TRY(dev_alloc(p, &p->pts, (size_t)J));
    SDP_TRY(dev_alloc(p, &p->tframe, (size_t)J));
    SDP_TRY(dev_alloc(p, &p->wts, (size_t)J * 3 * W));
    SDP_TRY(dev_alloc(p, &p->V, (size_t)d->T * Kz));
    if (d->flags & SDP_FLAG_BORROW_MAPS)
        p->S = const_cast<float2*>(static_cast<const float2*>(d->coil_maps));   // read only, caller-owned
    else
        SDP_TRY(dev_alloc(p, &p->S, (size_t)d->C * nvox));
    SDP_TRY(dev_alloc(p, &p->dinv, dinv.size()));
    SDP_TRY(dev_alloc(p, &p->tw, tw.size()));
    SDP_TRY(dev_alloc(p, &p->inc, inc.size()));
    SDP_TRY(dev_alloc(p, &p->subs, subs.size()));
    SDP_TRY(dev_alloc(p, &p->itiles, std::max<size_t>(itiles.size(), 1)));
    const size_t P = (size_t)bs[0] * bs[1] * bs[2];
    SDP_TRY(dev_alloc(p, &p->partials, (size_t)std::max(slots, 1LL) * P * Kz * p->maxB));
    SDP_TRY(dev_alloc(p, &p->counters, (size_t)nbins * p->maxB * ((K + 7) / 8)));
    SDP_TRY(dev_alloc(p, &p->status, 1));
    SDP_TRY(dev_alloc(p, &p->loss_partials, (size_t)residual_loss_partials(p->maxB, J)));
    SDP_TRY(dev_alloc(p, &p->loss_counter, 1));
    SDP_TRY(dev_alloc(p, &p->tv_part, (size_t)tv_partials(K, (int)p->n[0], (int)p->n[1], (int)p->n[2])));
    SDP_TRY(dev_alloc(p, &p->tv_counter, 1));
    const size_t before = p->total_bytes;
    const size_t gridA = (size_t)std::max<long long>(G, p->n[0] * p->n[1] * p->M[2]);
    const size_t gridB = (size_t)(p->n[0] * p->M[1] * p->M[2]);
    SDP_TRY(dev_alloc(p, &p->bufA, gridA * Kz * p->maxB));
    SDP_TRY(dev_alloc(p, &p->bufB, gridB * Kz * p->maxB));
    p->workspace_bytes = p->total_bytes - before;

    SDP_CUDA(cudaMemcpyAsync(p->pts, pts.data(), pts.size() * sizeof(float4), cudaMemcpyHostToDevice, st));
    SDP_CUDA(cudaMemcpyAsync(p->tframe, tf.data(), tf.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    SDP_CUDA(cudaMemcpyAsync(p->V, d->V, (size_t)d->T * Kz * sizeof(float2), cudaMemcpyDeviceToDevice, st));
    if (!(d->flags & SDP_FLAG_BORROW_MAPS))
        SDP_CUDA(cudaMemcpyAsync(p->S, d->coil_maps, (size_t)d->C * nvox * sizeof(float2), cudaMemcpyDeviceToDevice,
                                 st));
    SDP_CUDA(cudaMemcpyAsync(p->dinv, dinv.data(), dinv.size() * sizeof(float), cudaMemcpyHostToDevice, st));
    SDP_CUDA(cudaMemcpyAsync(p->tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice, st));
    SDP_CUDA(cudaMemcpyAsync(p->inc, inc.data(), inc.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    SDP_CUDA(cudaMemcpyAsync(p->subs, subs.data(), subs.size() * sizeof(SubProb), cudaMemcpyHostToDevice, st));
    if (!itiles.empty())
        SDP_CUDA(cudaMemcpyAsync(p->itiles, itiles.data(), itiles.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
    SDP_CUDA(cudaMemsetAsync(p->counters, 0, (size_t)nbins * p->maxB * ((K + 7) / 8) * sizeof(int), st));
    SDP_CUDA(cudaMemsetAsync(p->status, 0, sizeof(int), st));
    SDP_CUDA(cudaMemsetAsync(p->loss_counter, 0, sizeof(unsigned int), st));
    SDP_CUDA(cudaMemsetAsync(p->tv_counter, 0, sizeof(unsigned int), st));
    SDP_CUDA(launch_kb_weights(g, p->pts, p->wts, st));
    SDP_CUDA(cudaStreamSynchronize(st));
    size_t o = 0;
    for (int a = 0; a < 3; ++a) {
        p->ax[a].tw = p->tw + o;
        o += (size_t)g.M[a];
    }
    return SDP_OK;
}

// ---- profiling hooks ----
int prof_begin(sdp_plan_s* p, cudaStream_t st, ProfRec* rec) {
    if (!p->prof) return SDP_OK;
    if (p->prof_free.empty()) {
        ProfRec r;
        if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) {
            cudaGetLastError();
            return SDP_ERR_CUDA;
        }
        p->prof_free.push_back(r);
    }
    *rec = p->prof_free.back();
    p->prof_free.pop_back();
    SDP_CUDA(cudaEventRecord(rec->a, st));
    return SDP_OK;
}

int prof_end(sdp_plan_s* p, cudaStream_t st, ProfRec* rec, int stage) {
    if (!p->prof) return SDP_OK;
    rec->stage = stage;
    SDP_CUDA(cudaEventRecord(rec->b, st));
    p->prof_used.push_back(*rec);
    return SDP_OK;
}

template <typename F>
int run(sdp_plan_s* p, int stage, cudaStream_t st, F&& f) {
    ProfRec rec{};
    SDP_TRY(prof_begin(p, st, &rec));
    const cudaError_t e = f();
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SDP_ERR_CUDA;
    }
    return prof_end(p, st, &rec, stage);
}

const float* dinv_axis(const sdp_plan_s* p, int a) {
    size_t o = 0;
    for (int q = 0; q < a; ++q) o += (size_t)p->n[q];
    return p->dinv + o;
}

int check_call(const sdp_plan_s* p, const void* in, const int32_t* coil_idx, int B, int k0, int nk,
               const void* out) {
    if (!p || !in || !coil_idx || !out) return SDP_ERR_INVALID_ARG;
    if (B < 1 || B > p->maxB) return SDP_ERR_INVALID_ARG;
    if (k0 < 0 || nk < 1 || k0 + nk > p->geo.K) return SDP_ERR_INVALID_ARG;
    return SDP_OK;
}

// Whether step A3 of a call with nk channels runs the tiled interpolation: the plan
// asks for it, a kernel exists for the width and channel count, and every grid axis
// has at least 16 points (a tile with its margin then wraps around it at most once).
bool plan_interp_tiled(const sdp_plan_s* p, int nk) {
    const Geo& g = p->geo;
    return p->interp_tiled && interp_tiles_supported(g.W, nk) && g.M[0] >= 16 && g.M[1] >= 16 && g.M[2] >= 16;
}

// Step A3 of the plan: the tiled interpolation where the plan asks for it and a kernel
// exists for the width and channel count, else the row kernel.
cudaError_t plan_interp(const sdp_plan_s* p, const float2* grids, int B, int k0, int nk, float2* y, int accumulate,
                        cudaStream_t st) {
    const Geo& g = p->geo;
    if (plan_interp_tiled(p, nk))
        return launch_interp_tiles(g, p->itiles, p->n_itiles, p->nt[1], p->nt[2], p->pts, p->tframe, p->wts, p->V,
                                   grids, B, k0, nk, y, accumulate, p->status, p->wait_test_row, p->wait_test_ns, st);
    return launch_interp(g, p->interp_threads, p->interp_run, p->interp_coils, p->pts, p->tframe, p->wts, p->V, grids,
                         B, k0, nk, y, accumulate, st);
}

int forward_impl(sdp_plan_s* p, const void* x, const int32_t* coil_idx, int B, int k0, int nk, void* y,
                 int accumulate, cudaStream_t st) {
    SDP_TRY(check_call(p, x, coil_idx, B, k0, nk, y));
    const Geo& g = p->geo;
    const long long N1 = g.N[0], N2 = g.N[1];
    const long long M1 = g.M[0], M2 = g.M[1], M3 = g.M[2];
    const float2* xs = static_cast<const float2*>(x);
    SDP_TRY(run(p, ST_FWD_FFT3, st, [&] {
        return launch_fwd_prologue_fft3(g, p->ax[2], xs, p->S, coil_idx, B, k0, nk, dinv_axis(p, 0),
                                        dinv_axis(p, 1), dinv_axis(p, 2), p->bufA, p->status, st);
    }));
    SDP_TRY(run(p, ST_FWD_FFT2, st, [&] {
        return launch_fft_strided(p->ax[1], 0, p->bufA, p->bufB, (int)N2, 1, (int)M2, 0, M3 * nk, B * N1, st);
    }));
    SDP_TRY(run(p, ST_FWD_FFT1, st, [&] {
        return launch_fft_strided(p->ax[0], 0, p->bufB, p->bufA, (int)N1, 1, (int)M1, 0, M2 * M3 * nk, B, st);
    }));
    SDP_TRY(run(p, ST_INTERP, st, [&] {
        return plan_interp(p, p->bufA, B, k0, nk, static_cast<float2*>(y), accumulate, st);
    }));
    return SDP_OK;
}

int adjoint_impl(sdp_plan_s* p, const void* y, const int32_t* coil_idx, int B, int k0, int nk, void* out,
                 int accumulate, const float* scale, cudaStream_t st) {
    SDP_TRY(check_call(p, y, coil_idx, B, k0, nk, out));
    const Geo& g = p->geo;
    const long long N1 = g.N[0], N2 = g.N[1];
    const long long M1 = g.M[0], M2 = g.M[1], M3 = g.M[2];
    SDP_TRY(run(p, ST_SPREAD, st, [&] {
        return launch_spread(g, p->bs, p->nb, p->subs, p->nsub, p->inc, p->pts, p->tframe, p->wts, p->V,
                             static_cast<const float2*>(y), scale, B, k0, nk, p->bufA, p->partials, p->slots_per_b,
                             p->counters, p->nbins, p->spread_coils, st);
    }));
    SDP_TRY(run(p, ST_ADJ_FFT1, st, [&] {
        return launch_fft_strided(p->ax[0], 1, p->bufA, p->bufB, (int)M1, 0, (int)N1, 1, M2 * M3 * nk, B, st);
    }));
    SDP_TRY(run(p, ST_ADJ_FFT2, st, [&] {
        return launch_fft_strided(p->ax[1], 1, p->bufB, p->bufA, (int)M2, 0, (int)N2, 1, M3 * nk, B * N1, st);
    }));
    SDP_TRY(run(p, ST_ADJ_FFT3, st, [&] {
        return launch_adj_fft3_epilogue(g, p->ax[2], p->bufA, p->S, coil_idx, B, k0, nk, dinv_axis(p, 0),
                                        dinv_axis(p, 1), dinv_axis(p, 2), static_cast<float2*>(out), accumulate,
                                        p->status, st);
    }));
    return SDP_OK;
}

// ---- batched calls: a pool of worker streams and events per device ----
constexpr int kWorkers = 4;
constexpr int kMaxDevices = 64;
struct WorkerPool {
    bool ready = false;
    cudaStream_t st[kWorkers];
    cudaEvent_t fork;
    cudaEvent_t join[kWorkers];
};
std::mutex g_batch_mu;
WorkerPool g_pools[kMaxDevices];

int worker_pool(WorkerPool** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return SDP_ERR_CUDA;
    }
    WorkerPool& wp = g_pools[dev];
    if (!wp.ready) {
        for (int w = 0; w < kWorkers; ++w) {
            SDP_CUDA(cudaStreamCreateWithFlags(&wp.st[w], cudaStreamNonBlocking));
            SDP_CUDA(cudaEventCreateWithFlags(&wp.join[w], cudaEventDisableTiming));
        }
        SDP_CUDA(cudaEventCreateWithFlags(&wp.fork, cudaEventDisableTiming));
        wp.ready = true;
    }
    *out = &wp;
    return SDP_OK;
}

// ---- batched calls in one launch per stage (batch.cu) ----

// Whether the items can share launches: the same kernel width, channel count,
// spread bin shape and interpolation kernel (CTA size, tiled or not); one
// channel group (K <= 8 and K <= 32 / W); every grid length served by the
// two-pass FFT.
bool fused_eligible(const sdp_work* items, int n) {
    if (n < 1) return false;
    const sdp_plan_s* p0 = items[0].plan;
    for (int i = 0; i < n; ++i) {
        const sdp_plan_s* p = items[i].plan;
        if (p->geo.W != p0->geo.W || p->geo.K != p0->geo.K || p->bs[0] != p0->bs[0] || p->bs[2] != p0->bs[2] ||
            p->interp_threads != p0->interp_threads || p->interp_coils != p0->interp_coils ||
            p->interp_tiled != p0->interp_tiled)
            return false;
        if (p->geo.K > 8 || p->geo.K > 32 / p->geo.W || !mv_width_supported(p->geo.W)) return false;
        for (int a = 0; a < 3; ++a)
            if (p->ax[a].generic || !mv_length_supported(p->geo.M[a])) return false;
    }
    return true;
}

// One wave: items whose plans have room for all their coils at once.  Fills
// the launch descriptors and runs the four stages of one direction.
int run_wave(const sdp_work* items, const std::vector<int>& idx, const std::vector<int>& coil_off, bool adjoint,
             cudaStream_t st) {
    MvArgs a;
    std::memset(&a, 0, sizeof(a));
    const int n = (int)idx.size();
    const sdp_plan_s* p0 = items[idx[0]].plan;
    bool tiled = true;   // every item's interpolation tiled (the plans agree on asking for it)
    for (int q = 0; q < n; ++q) {
        const sdp_work& w = items[idx[q]];
        sdp_plan_s* p = w.plan;
        const Geo& g = p->geo;
        MvItem& it = a.it[q];
        const long long N1 = g.N[0], N2 = g.N[1];
        const long long M1 = g.M[0], M2 = g.M[1], M3 = g.M[2];
        const long long K = g.K;
        const size_t gridA = (size_t)std::max<long long>(M1 * M2 * M3, N1 * N2 * M3);
        const size_t gridB = (size_t)(N1 * M2 * M3);
        it.g = g;
        for (int d = 0; d < 3; ++d) {
            it.L[d] = g.M[d];
            it.tw[d] = p->ax[d].tw;
            it.d[d] = dinv_axis(p, d);
        }
        it.S = p->S;
        it.coil_idx = w.coil_idx;
        it.B = w.B;
        it.accumulate = w.accumulate ? 1 : 0;
        it.status = p->status;
        it.bufA = p->bufA + (size_t)coil_off[q] * gridA * K;
        it.bufB = p->bufB + (size_t)coil_off[q] * gridB * K;
        it.pts = p->pts;
        it.tframe = p->tframe;
        it.wts = p->wts;
        it.V = p->V;
        if (adjoint) {
            it.x = static_cast<float2*>(w.out);
            it.pass[0] = MvPass{it.bufA, it.bufB, (int)M1, 0, (int)N1, 1, M2 * M3 * K};
            it.pass[1] = MvPass{it.bufB, it.bufA, (int)M2, 0, (int)N2, 1, M3 * K};
        } else {
            it.x = const_cast<float2*>(static_cast<const float2*>(w.in));
            it.y = static_cast<float2*>(w.out);
            it.pass[1] = MvPass{it.bufA, it.bufB, (int)N2, 1, (int)M2, 0, M3 * K};
            it.pass[0] = MvPass{it.bufB, it.bufA, (int)N1, 1, (int)M1, 0, M2 * M3 * K};
        }
        SpreadArgs& sa = it.sa;
        sa.g = g;
        sa.bs1 = p->bs[0];
        sa.bs2 = p->bs[1];
        sa.bs3 = p->bs[2];
        sa.nb1 = p->nb[0];
        sa.nb2 = p->nb[1];
        sa.nb3 = p->nb[2];
        sa.subs = p->subs;
        sa.inc = p->inc;
        sa.pts = p->pts;
        sa.tframe = p->tframe;
        sa.wts = p->wts;
        sa.V = p->V;
        sa.y = adjoint ? static_cast<const float2*>(w.in) : nullptr;
        sa.scale = nullptr;
        sa.k0 = 0;
        sa.nk = g.K;
        sa.grids = it.bufA;
        sa.slot_elems = (long long)g.K * p->bs[0] * p->bs[1] * p->bs[2];
        sa.partials = p->partials + (size_t)coil_off[q] * (size_t)p->slots_per_b * (size_t)sa.slot_elems;
        sa.slots_per_b = p->slots_per_b;
        sa.counters = p->counters + (size_t)coil_off[q] * (size_t)p->nbins;
        sa.nbins = p->nbins;
        sa.ngroups = 1;
        sa.group = 0;
        it.nsub = p->nsub;
        it.spread_pairs = (spread_pairs_fit(p->bs[2], g.K) && p->spread_coils != 1 && w.B >= 2) ? 1 : 0;
        it.interp_coils = p->interp_coils > 0 && p->interp_coils < w.B ? p->interp_coils : w.B;
        it.itiles = p->itiles;
        it.n_itiles = p->n_itiles;
        it.nt2 = p->nt[1];
        it.nt3 = p->nt[2];
        tiled = tiled && plan_interp_tiled(p, g.K);
    }
    // units of each stage
    auto units = [&](auto count) {
        MvUnits u;
        u.n = n;
        u.start[0] = 0;
        for (int q = 0; q < n; ++q) u.start[q + 1] = u.start[q] + count(a.it[q]);
        return u;
    };
    auto ceil_div = [](long long x, long long y) { return (x + y - 1) / y; };
    const MvUnits u_fused_fwd = units([&](const MvItem& it) {
        return ceil_div((long long)it.g.N[0] * it.g.N[1] * it.g.K, mv_fused_lines(it.L[2])) * it.B;
    });
    const MvUnits u_fused_adj = units([&](const MvItem& it) {
        return ceil_div((long long)it.g.N[0] * it.g.N[1] * it.g.K, mv_fused_lines(it.L[2]));
    });
    auto u_strided = [&](int axis) {
        return units([&](const MvItem& it) {
            const long long outer = axis == 1 ? (long long)it.B * it.g.N[0] : (long long)it.B;
            return ceil_div(it.pass[axis].inner, mv_strided_cols(it.L[axis])) * outer;
        });
    };
    // stage timing (sdp_profile_*) is recorded on the first item's plan
    sdp_plan_s* pf = items[idx[0]].plan;
    if (!adjoint) {
        const MvUnits u2 = u_strided(1), u1 = u_strided(0);
        const MvUnits us = tiled ? units([&](const MvItem& it) { return (long long)it.n_itiles; })
                                 : units([&](const MvItem& it) { return (long long)it.g.J; });
        SDP_TRY(run(pf, ST_FWD_FFT3, st, [&] { return launch_mv_prologue(a, u_fused_fwd, st); }));
        SDP_TRY(run(pf, ST_FWD_FFT2, st, [&] { return launch_mv_strided(a, u2, 1, 0, st); }));
        SDP_TRY(run(pf, ST_FWD_FFT1, st, [&] { return launch_mv_strided(a, u1, 0, 0, st); }));
        SDP_TRY(run(pf, ST_INTERP, st, [&] {
            return tiled ? launch_mv_interp_tiles(a, us, p0->geo.W, p0->geo.K, st)
                         : launch_mv_interp(a, us, p0->geo.W, p0->interp_threads, st);
        }));
    } else {
        const MvUnits u1 = u_strided(0), u2 = u_strided(1);
        const MvUnits usp = units([&](const MvItem& it) {
            return (long long)it.nsub * (it.spread_pairs ? (it.B + 1) / 2 : it.B);
        });
        SDP_TRY(run(pf, ST_SPREAD, st, [&] { return launch_mv_spread(a, usp, p0->bs[0], p0->bs[2], p0->geo.W, p0->geo.K, st); }));
        SDP_TRY(run(pf, ST_ADJ_FFT1, st, [&] { return launch_mv_strided(a, u1, 0, 1, st); }));
        SDP_TRY(run(pf, ST_ADJ_FFT2, st, [&] { return launch_mv_strided(a, u2, 1, 1, st); }));
        SDP_TRY(run(pf, ST_ADJ_FFT3, st, [&] { return launch_mv_epilogue(a, u_fused_adj, st); }));
    }
    return SDP_OK;
}

// Bytes an item writes: y [B][J] (forward) or out [K][N1][N2][N3] (adjoint).
std::pair<uintptr_t, uintptr_t> out_range(const sdp_work& w, bool adjoint) {
    const sdp_plan_s* p = w.plan;
    const size_t n = adjoint ? (size_t)p->geo.K * p->n[0] * p->n[1] * p->n[2] : (size_t)w.B * p->geo.J;
    const uintptr_t a = reinterpret_cast<uintptr_t>(w.out);
    return {a, a + n * sizeof(float2)};
}

// Items in order; an item joins the current wave while its plan has room for
// its coils there (items of one plan take consecutive coil slices of the
// plan's workspace) and its output does not overlap the output of an item
// already in the wave (two items adding into one image must not run in the
// same launch), else the wave is run and a new one starts.
int run_batched_fused(const sdp_work* items, int n, bool adjoint, cudaStream_t st) {
    std::vector<int> idx, off;
    std::vector<std::pair<const sdp_plan_s*, int>> used;   // coils taken per plan in the wave
    for (int i = 0; i < n; ++i) {
        const sdp_plan_s* p = items[i].plan;
        int* u = nullptr;
        for (auto& e : used)
            if (e.first == p) u = &e.second;
        const int have = u ? *u : 0;
        const auto ri = out_range(items[i], adjoint);
        bool overlap = false;
        for (int q : idx) {
            const auto rq = out_range(items[q], adjoint);
            overlap |= ri.first < rq.second && rq.first < ri.second;
        }
        if ((int)idx.size() == kMaxMvItems || have + items[i].B > p->maxB || overlap) {
            SDP_TRY(run_wave(items, idx, off, adjoint, st));
            idx.clear();
            off.clear();
            used.clear();
            u = nullptr;
        }
        if (!u) {
            used.emplace_back(p, 0);
            u = &used.back().second;
        }
        idx.push_back(i);
        off.push_back(*u);
        *u += items[i].B;
    }
    if (!idx.empty()) SDP_TRY(run_wave(items, idx, off, adjoint, st));
    return SDP_OK;
}

int run_batched(const sdp_work* items, int n, bool adjoint, cudaStream_t st) {
    if (n < 0 || (n > 0 && !items)) return SDP_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i) {
        const sdp_work& w = items[i];
        if (!w.plan) return SDP_ERR_INVALID_ARG;
        SDP_TRY(check_call(w.plan, w.in, w.coil_idx, w.B, 0, w.plan->geo.K, w.out));
    }
    if (n == 0) return SDP_OK;
    if (fused_eligible(items, n) && !std::getenv("SDP_BATCH_STREAMS")) return run_batched_fused(items, n, adjoint, st);
    auto run_one = [&](const sdp_work& w, cudaStream_t s) {
        return adjoint ? adjoint_impl(w.plan, w.in, w.coil_idx, w.B, 0, w.plan->geo.K, w.out, w.accumulate ? 1 : 0,
                                      nullptr, s)
                       : forward_impl(w.plan, w.in, w.coil_idx, w.B, 0, w.plan->geo.K, w.out, 0, s);
    };
    // worker of each item: one worker per distinct plan (round robin), same plan -> same worker
    std::vector<sdp_plan_s*> plans;
    std::vector<int> worker(n);
    for (int i = 0; i < n; ++i) {
        int k = -1;
        for (size_t q = 0; q < plans.size(); ++q)
            if (plans[q] == items[i].plan) k = (int)q;
        if (k < 0) {
            k = (int)plans.size();
            plans.push_back(items[i].plan);
        }
        worker[i] = k % kWorkers;
    }
    if (plans.size() == 1) {   // nothing to overlap
        for (int i = 0; i < n; ++i) SDP_TRY(run_one(items[i], st));
        return SDP_OK;
    }
    std::lock_guard<std::mutex> lk(g_batch_mu);
    WorkerPool* wp = nullptr;
    SDP_TRY(worker_pool(&wp));
    const int used = (int)std::min<size_t>(plans.size(), kWorkers);
    SDP_CUDA(cudaEventRecord(wp->fork, st));
    for (int w = 0; w < used; ++w) SDP_CUDA(cudaStreamWaitEvent(wp->st[w], wp->fork, 0));
    int rc = SDP_OK;
    for (int i = 0; i < n && rc == SDP_OK; ++i) rc = run_one(items[i], wp->st[worker[i]]);
    // always join the workers back, also after a failed launch
    for (int w = 0; w < used; ++w) {
        if (cudaEventRecord(wp->join[w], wp->st[w]) != cudaSuccess ||
            cudaStreamWaitEvent(st, wp->join[w], 0) != cudaSuccess) {
            cudaGetLastError();
            rc = rc == SDP_OK ? SDP_ERR_CUDA : rc;
        }
    }
    return rc;
}

}  // namespace

extern "C" {

int sdp_forward_batched(const sdp_work* items, int32_t n, void* stream) {
    return run_batched(items, n, false, static_cast<cudaStream_t>(stream));
}

int sdp_adjoint_batched(const sdp_work* items, int32_t n, void* stream) {
    return run_batched(items, n, true, static_cast<cudaStream_t>(stream));
}

int sdp_plan_create(sdp_plan_t* out, const sdp_plan_desc* d, void* stream) {
    return sdp_plan_create_tuned(out, d, nullptr, stream);
}

int sdp_plan_create_tuned(sdp_plan_t* out, const sdp_plan_desc* d, const sdp_tuning* tn, void* stream) {
    if (!out) return SDP_ERR_INVALID_ARG;
    *out = nullptr;
    if (tn) {
        if (tn->spread_chunk < 32 || tn->spread_chunk > 65536 || tn->fft_engine < 0 || tn->fft_engine > 1 ||
            (tn->fft_lines != 0 && tn->fft_lines != 8 && tn->fft_lines != 4) ||
            (tn->fft_cols != 0 && tn->fft_cols != 32 && tn->fft_cols != 8) ||
            (tn->interp_threads != 0 && tn->interp_threads != 256 && tn->interp_threads != 1024) ||
            tn->spread_coils < 0 || tn->spread_coils > 2 ||
            (tn->interp_run != 0 && tn->interp_run != 1 && tn->interp_run != 2 && tn->interp_run != 4 &&
             tn->interp_run != 8) ||
            tn->interp_coils < 0 || tn->interp_coils > kMaxBatch || tn->fft_staged < 0 || tn->fft_staged > 3 ||
            tn->interp_tiled < 0 || tn->interp_tiled > 1)
            return SDP_ERR_INVALID_ARG;
        if (!spread_bins_supported(tn->spread_bins)) return SDP_ERR_UNSUPPORTED;
    }
    if (!d || !d->traj || !d->V || !d->coil_maps || !d->frame_offsets) return SDP_ERR_INVALID_ARG;
    for (int a = 0; a < 3; ++a)
        if (d->n[a] < 2) return SDP_ERR_INVALID_ARG;
    if (!(d->oversamp >= 1.0 && d->oversamp <= 4.0)) return SDP_ERR_INVALID_ARG;
    if (d->width < 2 || d->width > kMaxWidth) return SDP_ERR_UNSUPPORTED;
    if (d->K < 1 || d->K > kMaxK) return SDP_ERR_UNSUPPORTED;
    if (d->T < 1 || d->C < 1 || d->J < 1 || d->J >= (1LL << 31)) return SDP_ERR_INVALID_ARG;
    if (d->max_batch < 1 || d->max_batch > kMaxBatch) return SDP_ERR_INVALID_ARG;
    if (d->flags & ~(uint32_t)SDP_FLAG_BORROW_MAPS) return SDP_ERR_INVALID_ARG;
    if ((d->flags & SDP_FLAG_BORROW_MAPS) && (reinterpret_cast<uintptr_t>(d->coil_maps) % alignof(float2)))
        return SDP_ERR_INVALID_ARG;
    if (d->frame_offsets[0] != 0 || d->frame_offsets[d->T] != d->J) return SDP_ERR_INVALID_ARG;
    for (int t = 0; t < d->T; ++t)
        if (d->frame_offsets[t + 1] < d->frame_offsets[t]) return SDP_ERR_INVALID_ARG;
    // size limits, on the host before any device call: grid lengths up to 2^14, and one coil's
    // channel-interleaved grid and one image indexed with 32-bit offsets
    {
        long long G = 1, nvox = 1;
        for (int a = 0; a < 3; ++a) {
            const long long m = grid_len(d->n[a], d->oversamp, d->width);
            if (m > (1 << 14)) return SDP_ERR_UNSUPPORTED;
            G *= m;
            nvox *= d->n[a];
        }
        if (G * d->K >= (1LL << 31) || nvox >= (1LL << 31)) return SDP_ERR_UNSUPPORTED;
    }
    sdp_plan_s* p = new (std::nothrow) sdp_plan_s();
    if (!p) return SDP_ERR_OOM;
    if (cudaGetDevice(&p->dev) != cudaSuccess) {
        cudaGetLastError();
        delete p;
        return SDP_ERR_CUDA;
    }
    const int rc = build_plan(p, d, tn, static_cast<cudaStream_t>(stream));
    if (rc != SDP_OK) {
        free_plan(p);
        return rc;
    }
    *out = p;
    return SDP_OK;
}

void sdp_plan_destroy(sdp_plan_t p) { free_plan(p); }

int sdp_forward(sdp_plan_t p, const void* x, const int32_t* coil_idx, int32_t B, void* y, void* stream) {
    if (!p) return SDP_ERR_INVALID_ARG;
    return forward_impl(p, x, coil_idx, B, 0, p->geo.K, y, 0, static_cast<cudaStream_t>(stream));
}

int sdp_adjoint(sdp_plan_t p, const void* y, const int32_t* coil_idx, int32_t B, void* out, int32_t accumulate,
                void* stream) {
    if (!p) return SDP_ERR_INVALID_ARG;
    return adjoint_impl(p, y, coil_idx, B, 0, p->geo.K, out, accumulate ? 1 : 0, nullptr,
                        static_cast<cudaStream_t>(stream));
}

int sdp_adjoint_scaled(sdp_plan_t p, const void* y, const int32_t* coil_idx, int32_t B, const float* scale,
                       void* out, int32_t accumulate, void* stream) {
    if (!p || !scale) return SDP_ERR_INVALID_ARG;
    return adjoint_impl(p, y, coil_idx, B, 0, p->geo.K, out, accumulate ? 1 : 0, scale,
                        static_cast<cudaStream_t>(stream));
}

int sdp_residual_loss_weighted(sdp_plan_t p, const void* yhat, const void* y_meas, int32_t n_meas_rows,
                               const int32_t* meas_idx, int32_t B, const float* dcf, void* r2, float* loss,
                               void* stream) {
    if (!p || !yhat || !y_meas || !meas_idx || !r2 || !loss) return SDP_ERR_INVALID_ARG;
    if (B < 1 || B > p->maxB || n_meas_rows < 1) return SDP_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return run(p, ST_LOSS, st, [&] {
        return launch_residual_loss(static_cast<const float2*>(yhat), static_cast<const float2*>(y_meas), meas_idx,
                                    dcf, B, (long long)p->geo.J, n_meas_rows, static_cast<float2*>(r2),
                                    p->loss_partials, p->loss_counter, loss, p->status, st);
    });
}

int sdp_tv_value(sdp_plan_t p, const void* x, float eps, float lambda, float* value, void* stream) {
    if (!p || !x || !value || !(eps > 0.f)) return SDP_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return run(p, ST_TV, st, [&] {
        return launch_tv_value(p->geo, static_cast<const float2*>(x), eps, lambda, p->tv_part, p->tv_counter, value,
                               st);
    });
}

int sdp_tv_grad(sdp_plan_t p, const void* x, float eps, float lambda, const float* scale, void* out,
                int32_t accumulate, void* stream) {
    if (!p || !x || !out || !(eps > 0.f)) return SDP_ERR_INVALID_ARG;
    if (x == out) return SDP_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return run(p, ST_TV, st, [&] {
        return launch_tv_grad(p->geo, static_cast<const float2*>(x), eps, lambda, scale, static_cast<float2*>(out),
                              accumulate ? 1 : 0, st);
    });
}

int sdp_gram_samples(sdp_plan_t p, const void* y, int32_t B, void* out, void* stream) {
    if (!p || !y || !out || B < 1 || B > p->maxB) return SDP_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const Geo& g = p->geo;
    SDP_TRY(run(p, ST_SPREAD, st, [&] {
        return launch_spread(g, p->bs, p->nb, p->subs, p->nsub, p->inc, p->pts, p->tframe, p->wts, p->V,
                             static_cast<const float2*>(y), nullptr, B, 0, g.K, p->bufA, p->partials, p->slots_per_b,
                             p->counters, p->nbins, p->spread_coils, st);
    }));
    return run(p, ST_INTERP, st, [&] {
        return plan_interp(p, p->bufA, B, 0, g.K, static_cast<float2*>(out), 0, st);
    });
}

int sdp_residual_loss(sdp_plan_t p, const void* yhat, const void* y_meas, int32_t n_meas_rows,
                      const int32_t* meas_idx, int32_t B, void* r2, float* loss, void* stream) {
    return sdp_residual_loss_weighted(p, yhat, y_meas, n_meas_rows, meas_idx, B, nullptr, r2, loss, stream);
}

int sdp_forward_channels(sdp_plan_t p, const void* x, const int32_t* coil_idx, int32_t B, int32_t k0, int32_t nk,
                         void* y, int32_t accumulate, void* stream) {
    return forward_impl(p, x, coil_idx, B, k0, nk, y, accumulate ? 1 : 0, static_cast<cudaStream_t>(stream));
}

int sdp_adjoint_channels(sdp_plan_t p, const void* y, const int32_t* coil_idx, int32_t B, int32_t k0, int32_t nk,
                         void* out, int32_t accumulate, void* stream) {
    return adjoint_impl(p, y, coil_idx, B, k0, nk, out, accumulate ? 1 : 0, nullptr, static_cast<cudaStream_t>(stream));
}

int sdp_status(sdp_plan_t p, void* stream) {
    if (!p) return SDP_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return SDP_ERR_CUDA;
    }
    int v = 0;
    if (cudaMemcpy(&v, p->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemset(p->status, 0, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return SDP_ERR_CUDA;
    }
    return v;
}

int sdp_plan_info(sdp_plan_t p, int64_t* out, int32_t cap) {
    if (!p || !out || cap < 0) return SDP_ERR_INVALID_ARG;
    const int64_t v[16] = {p->M[0],        p->M[1],     p->M[2],   p->geo.J,
                           p->geo.K,       p->maxB,     p->bs[0],  p->bs[1],
                           p->bs[2],       p->nbins,    p->nsub,   p->ninc,
                           (int64_t)p->workspace_bytes, (int64_t)p->total_bytes, p->geo.W, p->geo.C};
    for (int i = 0; i < cap && i < 16; ++i) out[i] = v[i];
    return SDP_OK;
}

int sdp_plan_tuning(sdp_plan_t p, sdp_tuning* out) {
    if (!p || !out) return SDP_ERR_INVALID_ARG;
    *out = sdp_tuning{};
    for (int a = 0; a < 3; ++a) out->spread_bins[a] = p->bs[a];
    out->spread_chunk = p->spread_chunk;
    out->fft_engine = p->ax[0].generic;
    out->fft_lines = p->ax[2].lines;
    out->fft_cols = p->ax[0].cols;
    out->interp_threads = p->interp_threads;
    out->spread_coils = p->spread_coils;
    out->interp_run = p->interp_run;
    out->interp_coils = p->interp_coils;
    out->fft_staged = p->ax[2].staged;
    out->interp_tiled = p->interp_tiled;
    return SDP_OK;
}

double sdp_plan_beta(sdp_plan_t p) { return p ? p->beta : -1.0; }

size_t sdp_workspace_bytes(sdp_plan_t p) { return p ? p->workspace_bytes : 0; }

size_t sdp_workspace_bytes_for(sdp_plan_t p, int32_t maxB) {
    if (!p || maxB < 1 || maxB > kMaxBatch) return 0;
    const long long G = p->M[0] * p->M[1] * p->M[2];
    const size_t gridA = (size_t)std::max<long long>(G, p->n[0] * p->n[1] * p->M[2]);
    const size_t gridB = (size_t)(p->n[0] * p->M[1] * p->M[2]);
    return (gridA + gridB) * (size_t)p->geo.K * (size_t)maxB * sizeof(float2);
}

int sdp_plan_set_wait_test(sdp_plan_t p, int32_t withhold_row, int64_t timeout_ns) {
    if (!p) return SDP_ERR_INVALID_ARG;
    const int H = interp_tile_edge() + p->geo.W;
    if (withhold_row < -1 || withhold_row >= H * H) return SDP_ERR_INVALID_ARG;
    if (timeout_ns != 0 && (timeout_ns < 1000 || timeout_ns > 10000000000LL)) return SDP_ERR_INVALID_ARG;
    p->wait_test_row = withhold_row;
    p->wait_test_ns = timeout_ns;
    return SDP_OK;
}

int64_t sdp_launch_count(void) { return g_launches.load(); }

int sdp_profile_enable(sdp_plan_t p, int32_t enable) {
    if (!p) return SDP_ERR_INVALID_ARG;
    p->prof = enable != 0;
    return SDP_OK;
}

int sdp_profile_read(sdp_plan_t p, double* ms, int64_t* launches, int32_t cap) {
    if (!p) return -SDP_ERR_INVALID_ARG;
    for (auto& r : p->prof_used) {
        if (cudaEventSynchronize(r.b) != cudaSuccess) {
            cudaGetLastError();
            return -SDP_ERR_CUDA;
        }
        float t = 0.f;
        if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) {
            cudaGetLastError();
            return -SDP_ERR_CUDA;
        }
        p->prof_ms[r.stage] += t;
        p->prof_n[r.stage] += 1;
        p->prof_free.push_back(r);
    }
    p->prof_used.clear();
    const int n = cap < kNumStages ? cap : kNumStages;
    for (int s = 0; s < n; ++s) {
        if (ms) ms[s] = p->prof_ms[s];
        if (launches) launches[s] = p->prof_n[s];
        p->prof_ms[s] = 0;
        p->prof_n[s] = 0;
    }
    return n;
}

int64_t sdp_grid_size(int64_t n, double oversamp, int32_t width) {
    if (n < 1 || width < 2 || width > kMaxWidth || !(oversamp >= 1.0 && oversamp <= 4.0)) return -1;
    return grid_len(n, oversamp, width);
}

double sdp_kb_beta(int32_t width, double oversamp) {
    const double arg = (width / oversamp) * (width / oversamp) * (oversamp - 0.5) * (oversamp - 0.5) - 0.8;
    return arg > 0 ? kPi * std::sqrt(arg) : -1.0;
}

const char* sdp_strerror(int s) {
    switch (s) {
        case SDP_OK: return "ok";
        case SDP_ERR_INVALID_ARG: return "invalid argument";
        case SDP_ERR_OOM: return "device out of memory";
        case SDP_ERR_CUDA: return "CUDA runtime error";
        case SDP_ERR_TIMEOUT: return "bounded device wait timed out";
        case SDP_ERR_BOUNDS: return "device-side index out of range (coil index)";
        case SDP_ERR_UNSUPPORTED: return "unsupported parameters";
        default: return "unknown status";
    }
}

}  // extern "C"
