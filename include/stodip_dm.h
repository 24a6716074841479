/*
 * C ABI of MRF dictionary matching on sm_103a (GB300).
 *
 * Dictionary matching (StoDIP, Sec. 2 after Eq. 1; Ma et al. 2013, McGivney et
 * al. 2014) maps the reconstructed time-compressed image series (TSMI) to
 * quantitative maps by inverting the voxel-wise Bloch response
 * x_v = PD_v B(T1_v, T2_v): with the TSMI x_v in C^K of voxel v and the
 * temporally compressed dictionary atoms d_p in C^K (p = 0..P-1),
 *
 *     idx_v = argmax_p |d_p^H x_v| / ||d_p||,     PD_v = d_idx^H x_v / ||d_idx||^2,
 *
 * and T1_v, T2_v are the parameters of atom idx_v (the caller's table).  On
 * equal scores the lowest atom index wins; an atom of zero norm scores 0; a
 * zero voxel gets atom 0 and PD 0.
 *
 * How it is computed: the scores |d_p^H x_v|^2 / ||d_p||^2 of every (voxel,
 * atom) pair come from a tensor-core GEMM (tcgen05, fp16 operands, fp32
 * accumulation in tensor memory) of the unit-normalised voxels against the
 * unit-normalised atoms, with the real and imaginary parts of each inner
 * product as two output columns; its epilogue keeps, per voxel, the 32-atom
 * chunk holding the largest score.  A second pass recomputes that chunk's
 * inner products in float32 from the float32 inputs and takes the argmax and
 * PD there.  The chunk choice is therefore made at fp16 input precision
 * (|d^H x| of unit vectors to about 1e-3), the choice inside the chunk and PD
 * at float32 precision.
 *
 * All device pointers are CUDA device memory of the current device; all
 * sizes are element counts.  Calls are asynchronous on `stream` (a
 * cudaStream_t, NULL for the legacy default stream) and return SDP_OK or an
 * error code of stodip_op.h; none aborts or throws.
 */
#ifndef STODIP_DM_H
#define STODIP_DM_H

#include <stddef.h>
#include <stdint.h>

#include "stodip_op.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sdp_dm_s* sdp_dm_t;

/*
 * Build a matcher for the dictionary `atoms` (device, complex64 [P][K], row p =
 * atom d_p, read during the call only), with an optional parameter table
 * `params` (device float32 [P][2], (T1, T2) of atom p, copied; NULL for none),
 * for TSMIs of up to `max_vox` voxels.  1 <= K <= 16, 1 <= P <= 2^24, 1 <= max_vox <= 2^31 - 1, else
 * SDP_ERR_INVALID_ARG.  The matcher owns its device copies: the normalised
 * atoms in float32 and in the fp16 tile layout of the GEMM, 1/||d_p||, the
 * parameter table, and a
 * workspace of 2 * ceil(max_vox / 256) * 128 * 32 * ceil(2K / 16) bytes plus 16
 * bytes per voxel.  SDP_ERR_OOM when an allocation fails (nothing is leaked),
 * SDP_ERR_UNSUPPORTED on a device without tcgen05 (compute capability below
 * 10.0).  Synchronises `stream` before returning.
 */
int sdp_dm_create(sdp_dm_t* out, const void* atoms, const float* params, int64_t P, int32_t K,
                  int64_t max_vox, void* stream);

/* Release the matcher and its device memory (NULL is a no-op). */
void sdp_dm_destroy(sdp_dm_t dm);

/*
 * Match `nvox` voxels: x is device complex64 [K][nvox] (channel k of voxel v at
 * x[k * nvox + v], the TSMI layout [K][N1][N2][N3] flattened), idx is device
 * int32 [nvox], pd device complex64 [nvox]; both are written for every voxel.
 * qmap (device float32 [nvox][2], may be NULL) receives (T1, T2) of the matched
 * atom from the parameter table; non-NULL qmap without a table is
 * SDP_ERR_INVALID_ARG.  0 <= nvox <= max_vox, else SDP_ERR_INVALID_ARG (nvox = 0
 * launches nothing).
 * Launches 3 kernels; capturable in a CUDA graph.  The GEMM kernel bounds all
 * its waits (about one second each); if one gives up it records
 * SDP_ERR_TIMEOUT in the matcher's status word (read with sdp_dm_status) and
 * its outputs are not valid.
 */
int sdp_dm_match(sdp_dm_t dm, const void* x, int64_t nvox, int32_t* idx, void* pd, float* qmap, void* stream);

/*
 * Test hook for the bounded waits of the GEMM kernel (the paper has no
 * counterpart).  Every later sdp_dm_match of this matcher uses `timeout_ns`
 * as the limit of each mbarrier wait (0: the default of one second; else
 * 1e3 .. 1e10 ns), and, when withhold_tile >= 0, the first CTA's producer
 * never copies atom tile `withhold_tile` of its first voxel-tile pair: the
 * MMA threads' wait for that tile runs out, the kernel records SDP_ERR_TIMEOUT,
 * its CTA stops, waits (bounded) for the copies and MMAs it issued and frees
 * its tensor memory, and the match's outputs are not valid (they stay in
 * range).  withhold_tile = -1 turns the hook off.  Nothing faults or hangs:
 * this exercises the timeout path on the device.  SDP_ERR_INVALID_ARG for
 * withhold_tile outside [-1, atom tiles) or a limit out of range.
 */
int sdp_dm_set_wait_test(sdp_dm_t dm, int32_t withhold_tile, int64_t timeout_ns);

/* Synchronise `stream`, return the matcher's device status word and clear it. */
int sdp_dm_status(sdp_dm_t dm, void* stream);

/*
 * Matcher facts: writes min(cap, 8) int64 values
 *   [0] P  [1] K  [2] k-steps of 16 fp16 (ceil(2K / 16))  [3] atom tiles of 64
 *   [4] max_vox  [5] device bytes owned  [6] CTAs of the GEMM launch
 *   [7] tensor-core flops of one match per voxel (2 * 128 * 16 * k-steps per 64 atoms)
 * Returns SDP_OK or SDP_ERR_INVALID_ARG.
 */
int sdp_dm_info(sdp_dm_t dm, int64_t* out, int32_t cap);

#ifdef __cplusplus
}
#endif

#endif /* STODIP_DM_H */
