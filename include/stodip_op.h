/*
 * stodip_op.h -- C ABI of the GB300 (sm_103a) subspace multicoil NUFFT operator.
 *
 * StoDIP (arXiv 2408.02367), Sec. 2, Eq. 1: the acquisition operator A maps a
 * time-compressed image series x in C^{N x K} to multicoil non-Cartesian
 * k-space and "includes coil sensitivities, NUFFT and temporal SVD".  Sec. 2.1,
 * Eq. 3 splits it per coil, A = {A_c}, and Algorithm 1 applies one A_c (or a
 * minibatch of them) and its adjoint (through loss.backward()) per iteration.
 *
 * For a sample j of frame t_j at k-space location omega_j (radians):
 *
 *   A_c(x)[j] = sum_n exp(-i omega_j . n) S_c[n] sum_k V[t_j, k] x_k[n]
 *
 * with centred voxel indices n_d = i_d - floor(N_d / 2) (storage offset i_d).
 * The library evaluates this by Kaiser-Bessel gridding on a sigma-oversampled
 * grid of width-W kernels (Jackson et al. 1991; beta of Beatty et al. 2005):
 * deapodise and multiply by S_c, 3D FFT, interpolate W^3 taps contracting the K
 * channels with V[t_j, :].  The adjoint is the exact conjugate transpose of those
 * steps and sums over the coil minibatch (the gradient of sum_c L_c, Eq. 3).
 *
 * Conventions shared by every entry point
 *   - Complex values are interleaved float32 pairs (complex64), C order.
 *   - Every call returns an int status (SDP_OK = 0).  Nothing throws or aborts
 *     across the ABI.  Arguments are checked on the host before any launch;
 *     device-side faults of the data (a coil index out of range) are recorded in
 *     the plan's device status word and reported by sdp_status().
 *   - Pointers marked DEVICE must be CUDA device pointers on the plan's device;
 *     HOST pointers are ordinary host memory.  The caller owns every pointer it
 *     passes; the plan owns its own copies of V, S, the sorted trajectory, the
 *     bin tables and the workspace.
 *   - `stream` is a cudaStream_t passed as void* (0 = legacy default stream).
 *     sdp_forward / sdp_adjoint and their variants are asynchronous, allocate
 *     nothing and do not synchronise, so they can be captured in a CUDA graph.
 *   - Calls on one plan share its workspace: calls that overlap in time on
 *     different streams race.  Serialise them on one stream.
 */
#ifndef STODIP_OP_H
#define STODIP_OP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define SDP_OK 0
#define SDP_ERR_INVALID_ARG 1   /* bad pointer, size or parameter (checked on the host) */
#define SDP_ERR_OOM 2           /* device allocation failed in sdp_plan_create */
#define SDP_ERR_CUDA 3          /* a CUDA runtime call failed */
#define SDP_ERR_TIMEOUT 4       /* a bounded device wait gave up */
#define SDP_ERR_BOUNDS 5        /* device-side index check failed (coil index) */
#define SDP_ERR_UNSUPPORTED 6   /* parameters outside the supported range */

/*
 * Plan flags (bit mask).
 *   SDP_FLAG_BORROW_MAPS  the plan keeps the caller's coil_maps pointer instead
 *                         of copying the maps (C x N1 N2 N3 x 8 bytes: 1.6 GB for
 *                         32 coils at 200 x 200 x 160).  The caller keeps that
 *                         DEVICE buffer alive and unchanged until
 *                         sdp_plan_destroy; kernels only read it.
 * Other bits are reserved: a plan whose flags hold one gets SDP_ERR_INVALID_ARG.
 * (The spread is always deterministic, bitwise: every grid point is written
 * exactly once; and the adjoint never needs the forward's grid, so the plan has
 * nothing to recompute.  Neither needs a flag.)
 */
#define SDP_FLAG_NONE 0u
#define SDP_FLAG_BORROW_MAPS 1u

/* Opaque plan, owned by the library. */
typedef struct sdp_plan_s* sdp_plan_t;

/*
 * Description of one operator (one trajectory, one image matrix).
 *   n[3]           image matrix N1, N2, N3 (axis 3 contiguous), each >= 2.
 *   oversamp       grid oversampling sigma in [1, 4]; the grid length along axis d
 *                  is the smallest even 2,3,5-smooth M_d >= max(ceil(sigma N_d), 2W).
 *                  M1 M2 M3 K < 2^31 (the K channel grids of one coil, interleaved
 *                  per grid point, are indexed with 32-bit offsets), N1 N2 N3 < 2^31
 *                  and every M_d <= 2^14, else SDP_ERR_UNSUPPORTED, returned on
 *                  the host before any device call or read of traj, V or coil_maps.
 *   width          Kaiser-Bessel kernel width W in taps, 2..8.
 *   K              subspace rank (channels of x), 1..16.
 *   T              frames (rows of V), >= 1.
 *   C              coils (rows of coil_maps), >= 1.
 *   J              samples per coil (all frames), >= 1 and < 2^31.
 *   max_batch      largest coil minibatch B of any later call, 1..64; the
 *                  workspace is sized for it.
 *   frame_offsets  HOST int64 [T+1]: samples of frame t are [off[t], off[t+1]),
 *                  off[0] = 0, off[T] = J, non-decreasing.  Read during create only.
 *   traj           DEVICE float32 [J][3], omega in radians, |omega_d| <= pi;
 *                  omega[:, d] pairs with image axis d.  Read during create only.
 *   V              DEVICE complex64 [T][K] temporal subspace basis, copied.
 *   coil_maps      DEVICE complex64 [C][N1][N2][N3] coil sensitivities S_c, copied
 *                  (or borrowed, with SDP_FLAG_BORROW_MAPS).
 *   flags          SDP_FLAG_NONE or SDP_FLAG_BORROW_MAPS.
 */
typedef struct {
    int64_t n[3];
    double oversamp;
    int32_t width;
    int32_t K;
    int32_t T;
    int32_t C;
    int64_t J;
    int32_t max_batch;
    uint32_t flags;
    const int64_t* frame_offsets;
    const float* traj;
    const void* V;
    const void* coil_maps;
} sdp_plan_desc;

/*
 * Build a plan: grid sizes, Kaiser-Bessel beta and deapodisation tables, FFT
 * twiddles (float64 on the host, stored as float32), grid coordinates of every
 * sample, the bin sort of the samples and the bin incidence lists of the
 * adjoint, copies of V and S, and a workspace for max_batch coils.
 * Allocates device memory and synchronises `stream`; not capturable.
 * On success *out holds the plan; on failure *out is NULL and nothing leaks.
 */
int sdp_plan_create(sdp_plan_t* out, const sdp_plan_desc* desc, void* stream);

/*
 * Kernel-shape choices of a plan, for an autotuner (the paper has no
 * counterpart: it leaves the NUFFT's internals to a library).  Every choice
 * computes the same operator; they differ in speed and in the order of
 * floating-point sums only.
 *   spread_bins   grid points per spread bin (axis 1, 2, 3): {8, 4, 8} (default,
 *                 a lane per 8-point axis-3 column), {8, 4, 4} (half-depth
 *                 columns: fewer registers per lane, more incidences per sample),
 *                 {4, 4, 8} or {4, 4, 4} (16 columns, two lanes per column, the
 *                 two half-warps taking alternate incidences).
 *   spread_chunk  incidences per spread subproblem, 32 .. 65536 (default 512):
 *                 bounds the work of one CTA on the dense k-space centre.
 *   fft_engine    0: two-pass register FFTs where the length has one (default),
 *                 1: the radix-2/3/4/5 Stockham kernels for every length.
 *   fft_lines     grid lines per CTA of the fused axis-3 FFT kernels (the
 *                 forward prologue and the adjoint epilogue): 0 (default: 16,
 *                 or 8 for lengths >= 240), 8 or 4 (fewer lines: more, smaller
 *                 CTAs, so more of them resident per SM).
 *   fft_cols      grid columns per CTA of the strided axis-1 and axis-2 FFT
 *                 passes: 0 (default: 16), 32 (lengths up to 160; longer axes
 *                 keep the default) or 8.
 *   interp_threads  threads per CTA of the persistent interpolation kernel:
 *                 0 (default: 256), 256 or 1024 (W <= 4 only, else
 *                 SDP_ERR_UNSUPPORTED).  1024 puts one CTA on an SM, whose
 *                 warps then gather for consecutive samples and share the SM's
 *                 L1; it can pay for a minibatch of one or two coils and loses
 *                 badly for eight (the L1 holds fewer coils' windows).
 *   spread_coils  coils of the minibatch one spread warp accumulates: 0 (default:
 *                 two where the doubled register columns fit, i.e. 4-deep bins
 *                 with at most 5 channels per group, else one), 1 or 2 (2 falls
 *                 back to one where it does not fit).  Two coils share one
 *                 staging of each incidence's positions and weights.
 *   interp_run    consecutive bin-sorted samples one interpolation warp takes
 *                 before it jumps ahead by the whole grid of warps: 0 (default:
 *                 1), 1, 2, 4 or 8.  Longer runs let a warp's next sample find
 *                 its window rows in the SM's L1.
 *   interp_coils  coils of the minibatch per sweep of the interpolation over
 *                 the samples: 0 (default: all of them, each sample's window
 *                 set up once) or 1 .. 64 (e.g. 2: the samples are swept B / 2
 *                 times, each sweep gathering from two coils' grids only, which
 *                 keeps a large minibatch's working set within L2 and the TLB).
 *   fft_staged    fused axis-3 kernels with their inputs staged by bulk copies
 *                 (cp.async.bulk into double-buffered shared memory, persistent
 *                 CTAs, whole image rows per unit), a bit mask: 1 the forward
 *                 prologue, 2 the adjoint epilogue, 3 both, 0 (default) neither.
 *                 Where a staged kernel does not apply (a two-pass length, even
 *                 N3 and 16-byte aligned inputs are needed) the direct-load
 *                 kernel runs.  Other values: SDP_ERR_INVALID_ARG.
 *   interp_tiled  interpolation from shared-memory tiles: 0 (default: off, the
 *                 row kernel) or 1 (on where supported: W = 2 or 4 and at most 8
 *                 channels per call; elsewhere the row kernel).  The plan orders
 *                 the samples by tiles of 8^3 grid points either way; the tiled
 *                 kernel copies each tile's grid with its window margin into
 *                 shared memory once per coil and interpolates the tile's samples
 *                 from there.  The batched calls run tiled plans with the same
 *                 tile kernel, one launch over the work items of every plan.
 */
typedef struct {
    int32_t spread_bins[3];
    int32_t spread_chunk;
    int32_t fft_engine;
    int32_t fft_lines;
    int32_t fft_cols;
    int32_t interp_threads;
    int32_t spread_coils;
    int32_t interp_run;
    int32_t interp_coils;
    int32_t fft_staged;
    int32_t interp_tiled;
} sdp_tuning;

/*
 * sdp_plan_create with the kernel shapes of `tuning` (NULL: the defaults, with
 * the SDP_SPREAD_CHUNK and SDP_FFT_GENERIC environment overrides honoured).
 * SDP_ERR_UNSUPPORTED for a bin shape without a kernel, SDP_ERR_INVALID_ARG
 * for other values out of range (checked on the host before any device work).
 */
int sdp_plan_create_tuned(sdp_plan_t* out, const sdp_plan_desc* desc, const sdp_tuning* tuning, void* stream);

/* The kernel shapes a plan was built with (SDP_OK or SDP_ERR_INVALID_ARG). */
int sdp_plan_tuning(sdp_plan_t plan, sdp_tuning* out);

/* Release every resource of the plan (NULL is a no-op).  Synchronises the device. */
void sdp_plan_destroy(sdp_plan_t plan);

/*
 * Forward operator on a coil minibatch (Eq. 1 / Eq. 3, Algorithm 1 line 4):
 *   y[b][j] = A_{coil_idx[b]}(x)[j]   for b < B, j < J.
 *   x         DEVICE complex64 [K][N1][N2][N3]
 *   coil_idx  DEVICE int32 [B], each in [0, C); duplicates allowed.  Read by the
 *             kernels, so a captured graph sees the values present at replay.
 *   B         1..max_batch
 *   y         DEVICE complex64 [B][J] (overwritten)
 */
int sdp_forward(sdp_plan_t plan, const void* x, const int32_t* coil_idx, int32_t B,
                void* y, void* stream);

/*
 * Adjoint on a coil minibatch, summed over it (the gradient of
 * sum_{b} L_{c_b}, Eq. 3, as used by loss.backward() in Algorithm 1):
 *   out_k = (accumulate ? out_k : 0) + sum_b A_{coil_idx[b]}^H (y[b])   (channel k)
 *   y         DEVICE complex64 [B][J]
 *   coil_idx  DEVICE int32 [B] as in sdp_forward
 *   out       DEVICE complex64 [K][N1][N2][N3]
 *   accumulate 0 = overwrite, 1 = add into out
 */
int sdp_adjoint(sdp_plan_t plan, const void* y, const int32_t* coil_idx, int32_t B,
                void* out, int32_t accumulate, void* stream);

/*
 * Channel-range forms of the two calls (the building block of the plain
 * one-coil-one-channel-per-launch form, and of callers that split K):
 *   forward: y[b] = (accumulate ? y[b] : 0) + sum_{k0 <= k < k0+nk} V[t_j,k] NUFFT(S_c x_k)
 *   adjoint: out_k (+)= sum_b A^H restricted to channel k, for k0 <= k < k0+nk only;
 *            other channels of out are not touched.
 *   0 <= k0, 1 <= nk, k0 + nk <= K.
 */
int sdp_forward_channels(sdp_plan_t plan, const void* x, const int32_t* coil_idx, int32_t B,
                         int32_t k0, int32_t nk, void* y, int32_t accumulate, void* stream);
int sdp_adjoint_channels(sdp_plan_t plan, const void* y, const int32_t* coil_idx, int32_t B,
                         int32_t k0, int32_t nk, void* out, int32_t accumulate, void* stream);

/*
 * Adjoint with the input scaled by a DEVICE float32 scalar:
 *   out_k = (accumulate ? out_k : 0) + (*scale) * sum_b A_{coil_idx[b]}^H (y[b]).
 * The scale is read by the kernel, so an autograd backward can pass the
 * incoming gradient of a scalar loss without a host synchronisation.
 */
int sdp_adjoint_scaled(sdp_plan_t plan, const void* y, const int32_t* coil_idx, int32_t B, const float* scale,
                       void* out, int32_t accumulate, void* stream);

/*
 * Data-consistency residual and loss of Eq. 3 (DCF = 1), Algorithm 1 line 5,
 * summed over the minibatch:
 *   r2[b][j] = 2 (yhat[b][j] - y_meas[meas_idx[b]][j])   (dL/dyhat, PyTorch convention)
 *   *loss    = sum_b sum_j |yhat[b][j] - y_meas[meas_idx[b]][j]|^2
 *   yhat      DEVICE complex64 [B][J]
 *   y_meas    DEVICE complex64 [n_meas_rows][J] (e.g. all C coils, or one row per b)
 *   meas_idx  DEVICE int32 [B], rows of y_meas, each in [0, n_meas_rows)
 *   r2        DEVICE complex64 [B][J] (overwritten)
 *   loss      DEVICE float32 scalar (overwritten).  Each thread adds the
 *             |r|^2 of its 4 entries and each warp its 128 entries in float32;
 *             the warps of a block and then the blocks are added in float64,
 *             every sum in a fixed order, so the loss is bitwise repeatable.
 */
int sdp_residual_loss(sdp_plan_t plan, const void* yhat, const void* y_meas, int32_t n_meas_rows,
                      const int32_t* meas_idx, int32_t B, void* r2, float* loss, void* stream);

/*
 * Density-compensated data-consistency loss (Sec. 2, Eq. 2: ||sqrt(DCF) y -
 * sqrt(DCF) A(x)||^2, per coil Eq. 3), the form sdp_residual_loss takes with
 * DCF = 1:
 *   r2[b][j] = 2 dcf[j] (yhat[b][j] - y_meas[meas_idx[b]][j])
 *   *loss    = sum_b sum_j dcf[j] |yhat[b][j] - y_meas[meas_idx[b]][j]|^2
 *   dcf      DEVICE float32 [J] per-sample weights (shared by all coils), or
 *            NULL for 1.  Other arguments as in sdp_residual_loss.
 */
int sdp_residual_loss_weighted(sdp_plan_t plan, const void* yhat, const void* y_meas, int32_t n_meas_rows,
                               const int32_t* meas_idx, int32_t B, const float* dcf, void* r2, float* loss,
                               void* stream);

/*
 * Sample-domain Gram of the gridding interpolator with the subspace folded in:
 *   out[b][j] = sum_k V[t_j,k] sum_m phi(g_j - m) sum_i phi(g_i - m) conj(V[t_i,k]) y[b][i]
 * i.e. the interpolation step applied to the spread step, without FFT,
 * deapodisation or coil maps.  With K = 1 and V = 1 it is the
 * Phi Phi^H of the iterative density compensation of Pipe & Menon 1999,
 * w <- w / (Phi Phi^H w), which gives the DCF of Eq. 2 (the paper names a DCF
 * without saying how it is computed).
 *   y, out  DEVICE complex64 [B][J], 1 <= B <= max_batch; uses the workspace.
 */
int sdp_gram_samples(sdp_plan_t plan, const void* y, int32_t B, void* out, void* stream);

/*
 * Spatial total variation of the TSMI, the penalty of Algorithm 1 line 6
 * (loss = L_c + lambda TV(x_hat), Sec. 2.1).  The paper does not define TV;
 * this is the isotropic TV of every subspace channel with smoothing eps > 0,
 * forward differences D_d and a zero difference at the last index of an axis:
 *   TV(x) = sum_k sum_n sqrt(|D1 x_k(n)|^2 + |D2 x_k(n)|^2 + |D3 x_k(n)|^2 + eps^2)
 *   x      DEVICE complex64 [K][N1][N2][N3] (the plan's image size)
 *   value  DEVICE float32 scalar: lambda TV(x), accumulated in float64, fixed order
 *   out    DEVICE complex64 [K][N1][N2][N3]:
 *          (accumulate ? out : 0) + lambda (*scale) (dTV/dRe + i dTV/dIm)
 *   scale  DEVICE float32 scalar or NULL (1); out must not alias x.
 */
int sdp_tv_value(sdp_plan_t plan, const void* x, float eps, float lambda, float* value, void* stream);
int sdp_tv_grad(sdp_plan_t plan, const void* x, float eps, float lambda, const float* scale, void* out,
                int32_t accumulate, void* stream);

/*
 * One application of an operator inside a batch (several volumes / plans):
 *   plan      the item's plan
 *   in        forward: DEVICE x [K][N1][N2][N3]; adjoint: DEVICE y [B][J]
 *   coil_idx  DEVICE int32 [B]
 *   B         1..max_batch of the plan
 *   accumulate forward: ignored (y is overwritten); adjoint: 0 overwrite, 1 add
 *   out       forward: DEVICE y [B][J]; adjoint: DEVICE out [K][N1][N2][N3]
 */
typedef struct {
    sdp_plan_t plan;
    const void* in;
    const int32_t* coil_idx;
    int32_t B;
    int32_t accumulate;
    void* out;
} sdp_work;

/*
 * Apply the forward (resp. adjoint) operator of every item (StoDIP Eq. 3 for
 * several reconstructions at once, e.g. uneven coil minibatches of volumes of
 * different matrix sizes).  All items are checked before anything is launched.
 *
 * One launch per stage: when every item's plan has the same kernel width W
 * (4 or 6), channel count K (K <= 8 and K <= 32 / W), spread bin depth and
 * interpolation CTA size, and every grid length has a two-pass FFT (48, 64,
 * 80, 96, 100, 120, 128, 160, 200, 240, 250, 256), the whole batch is one
 * launch per stage: 4 for the forward (prologue + axis-3 FFT, axis-2 FFT,
 * axis-1 FFT, interpolation), 4 for the adjoint (spread, inverse axis-1 and
 * axis-2 FFTs, axis-3 FFT + epilogue), each covering the work of every item.
 * Items that share a plan take consecutive coil slices of its workspace; when
 * their minibatches together exceed its max_batch, or when an item's output
 * overlaps the output of an earlier item of the batch (e.g. two adjoints
 * adding into one image), the batch runs in waves of such launch sets, in item
 * order.  These launches are on `stream` itself.  Up to 16 items per wave.
 *
 * Otherwise (or with the environment variable SDP_BATCH_STREAMS set) each
 * item runs its own launches: items whose plans differ run concurrently on
 * library-owned worker streams forked from and joined back to `stream`, items
 * that share a plan one after the other.  The worker streams of a device are
 * created by its first such call: make that call before any stream capture.
 *
 * Either way the whole batch is ordered after earlier work on `stream` and
 * before later work on it, and can be captured in a CUDA graph.  Batched
 * calls from several host threads are serialised by the library.
 */
int sdp_forward_batched(const sdp_work* items, int32_t n, void* stream);
int sdp_adjoint_batched(const sdp_work* items, int32_t n, void* stream);

/*
 * Residual and loss of sdp_residual_loss without a plan and without any device
 * allocation.  The paper has no counterpart: this exists for callers that
 * cannot call cudaMalloc (device memory owned by a host framework whose
 * allocator must account for every byte, a process under a hard memory cap,
 * or work recorded while allocation is forbidden), who therefore cannot
 * create a plan.
 *   It computes what sdp_residual_loss computes, i.e. sdp_residual_loss_weighted
 *   with dcf = NULL: there is no density compensation (every sample weight 1).
 *   yhat, y_meas, meas_idx, r2, loss: as in sdp_residual_loss (DEVICE);
 *   B >= 1 rows of yhat, J >= 1 samples per row, B * J <= SDP_NOALLOC_MAX_ELEMS,
 *   larger sizes return SDP_ERR_INVALID_ARG.  Rows of meas_idx outside
 *   [0, n_meas_rows) contribute a zero residual and raise no SDP_ERR_BOUNDS
 *   (there is no status word).  |r|^2 is added in float32 four entries at a
 *   time per thread and in float64 from there on, in a fixed order.
 * Scratch: a fixed 32 KB + 256 B array inside the library image on every
 * device that loads the library, held until the process exits.  The first
 * call on a device looks its address up (cudaGetSymbolAddress, with that
 * device current); make that first call before any stream capture.  All calls
 * on a device share the array, so calls that overlap on the GPU race: the
 * caller serialises them.  Each call clears the completion counter before
 * its kernel and rewrites every partial sum it reads.
 */
#define SDP_NOALLOC_MAX_ELEMS (1LL << 28)
int sdp_residual_loss_noalloc(const void* yhat, const void* y_meas, int32_t n_meas_rows,
                              const int32_t* meas_idx, int32_t B, int64_t J, void* r2, float* loss,
                              void* stream);

/*
 * Synchronise `stream`, return the plan's device status word (SDP_OK or the
 * first device-side error recorded since the last call) and clear it.
 */
int sdp_status(sdp_plan_t plan, void* stream);

/*
 * Plan facts for callers and tests.  Writes min(cap, 16) int64 values:
 *   [0..2] grid M1, M2, M3   [3] J   [4] K   [5] max_batch
 *   [6..8] spread bin sizes  [9] number of bins  [10] number of spread subproblems
 *   [11] incidences (sample, bin) of the adjoint  [12] workspace bytes
 *   [13] plan-owned device bytes in total  [14] width W  [15] C
 * Returns SDP_OK or SDP_ERR_INVALID_ARG.
 */
int sdp_plan_info(sdp_plan_t plan, int64_t* out, int32_t cap);

/* Kaiser-Bessel beta the plan uses (Beatty et al. 2005), or -1 for a NULL plan. */
double sdp_plan_beta(sdp_plan_t plan);

/* Bytes of device workspace the plan holds for its max_batch (0 for NULL). */
size_t sdp_workspace_bytes(sdp_plan_t plan);

/*
 * Bytes of device workspace a plan of the same geometry, trajectory and kernel
 * shapes would hold for a coil minibatch of up to maxB coils (1..64), for
 * callers that size several plans against a memory budget; 0 for a NULL plan or
 * maxB out of range.  Host only, no device work.
 */
size_t sdp_workspace_bytes_for(sdp_plan_t plan, int32_t maxB);

/*
 * Test hook for the bounded waits of the tiled interpolation (interp_tiled;
 * the paper has no counterpart).  While withhold_row >= 0, every later forward
 * of this plan that runs the tiled kernel has its first CTA not copy row
 * withhold_row (0 .. (8 + W)^2 - 1) of its first tile for the first coil: that
 * CTA's wait for the tile runs out after timeout_ns (0: the default of one
 * second; else 1e3 .. 1e10 ns), it records SDP_ERR_TIMEOUT in the status word,
 * waits once more (bounded) and leaves, and the forward's output is not valid.
 * withhold_row = -1 turns the hook off (the limit stays).  Nothing faults or
 * hangs: this exercises the timeout path on the device.  SDP_ERR_INVALID_ARG
 * for a NULL plan or a value out of range.
 */
int sdp_plan_set_wait_test(sdp_plan_t plan, int32_t withhold_row, int64_t timeout_ns);

/* Kernels launched by this library in this process so far (all plans). */
int64_t sdp_launch_count(void);

/*
 * Per-stage timing with CUDA events on the launching stream.
 * sdp_profile_enable(plan, 1) brackets every later launch of the plan with a
 * pair of events (recorded on the launch's own stream); sdp_profile_read
 * synchronises those events, adds each launch's duration to its stage and
 * writes up to `cap` stages: ms[s] = summed milliseconds, launches[s] = count.
 * Stages: 0 prologue+FFT axis 3, 1 FFT axis 2, 2 FFT axis 1, 3 interpolation,
 * 4 spread, 5 inverse FFT axis 1, 6 inverse FFT axis 2, 7 inverse FFT axis 3
 * + epilogue, 8 residual and loss, 9 total variation.  Reading resets the sums.  Returns the number of stages written
 * or a negative status.  Profiling is off by default and costs two event
 * records per launch when on.
 */
int sdp_profile_enable(sdp_plan_t plan, int32_t enable);
int sdp_profile_read(sdp_plan_t plan, double* ms, int64_t* launches, int32_t cap);

/*
 * Host-only helpers (no device, no plan), for callers that size buffers:
 *   sdp_grid_size: the oversampled grid length a plan uses for an axis of n
 *                  voxels, the smallest even 2,3,5-smooth M >= max(ceil(sigma n), 2W);
 *                  -1 for n < 1, W outside 2..8 or sigma outside [1, 4].
 *   sdp_kb_beta:   the Kaiser-Bessel shape parameter of width W and oversampling
 *                  sigma, pi sqrt((W/sigma)^2 (sigma - 1/2)^2 - 0.8) (Beatty et al.
 *                  2005); -1 when the square root's argument is not positive.
 */
int64_t sdp_grid_size(int64_t n, double oversamp, int32_t width);
double sdp_kb_beta(int32_t width, double oversamp);

/* Static text for a status code. */
const char* sdp_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* STODIP_OP_H */
