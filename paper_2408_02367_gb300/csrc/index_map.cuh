// Index maps of the channel-interleaved kernels: which lane or thread of a
// kernel touches which element of which buffer.  Plain integer arithmetic kept
// in one place, compiled into the kernels and, for the tests, into a host
// library that enumerates every map over many shapes and checks that each
// element is written (or read) exactly once, that every index stays inside its
// buffer, and that the spread's 16-byte shared-memory accesses of a
// quarter-warp meet distinct banks.  Nothing here is method arithmetic.
#pragma once

#if defined(__CUDACC__)
#define SDP_MAP __host__ __device__ __forceinline__
#else
#define SDP_MAP inline
#endif

namespace sdp {
namespace imap {

// ---------------- adjoint spread (spread_impl.cuh) ----------------
// A bin has ncol = B1 x 4 columns; a column holds B3 points x nk channels of
// (Re, Im) values, i.e. CQ = B3 nk / 2 16-byte pairs (B3 is a multiple of 4).
// In the shared transposition buffer column slot cl starts at pair cl TS, with
// TS = CQ | 1: an odd stride, so the 16-byte accesses of a quarter-warp to
// consecutive column slots fall on distinct banks.
SDP_MAP constexpr int spread_cq(int B3, int nk) { return B3 * nk / 2; }
SDP_MAP constexpr int spread_ts(int B3, int nk) { return (B3 * nk / 2) | 1; }

// Register-to-shared transposition: with ipw incidences per warp step, the
// lanes of incidence slot h (lane / ncol) write the pairs j with j % ipw == h
// of their column; with one incidence per step a lane writes every pair.
SDP_MAP constexpr bool spread_owns_pair(int j, int ipw, int h) { return ipw == 1 || j % ipw == h; }

// Column slot cl = s ncol + c: coil slot s of the warp, column c = (c1, c2) =
// (c / 4, c % 4) of the bin.
struct SpreadPiece {
    int cl, s, c, c1, c2, j;
};

// Piece e of a store of whole columns (all channels of the grid in the call):
// 16-byte pair j of column slot cl, the warp's lanes taking e = lane, lane + 32, ...
SDP_MAP SpreadPiece spread_pair_piece(int e, int cq, int ncol) {
    const int cl = e / cq, j = e - cl * cq;
    const int s = cl / ncol, c = cl % ncol;
    return {cl, s, c, c >> 2, c & 3, j};
}

// Piece e of a store of one channel group (nkt channels of a grid with more):
// 8-byte value r = x3 nkt + q of column slot cl, per = B3 nkt values a column.
struct SpreadValue {
    int cl, s, c1, c2, x3, q, r;
};

SDP_MAP SpreadValue spread_value_piece(int e, int per, int nkt, int ncol) {
    const int cl = e / per, r = e - cl * per;
    const int x3 = r / nkt, q = r - x3 * nkt;
    const int s = cl / ncol, c = cl % ncol;
    return {cl, s, c >> 2, c & 3, x3, q, r};
}

// The last chunk of a multi-chunk bin sums the partial tiles: piece e is column
// c = e % ncol (fastest, so a warp reads contiguous 16-byte pairs of a partial),
// then pair j, then coil slot s.
SDP_MAP SpreadPiece spread_sum_piece(int e, int cq, int ncol) {
    const int c = e % ncol, cj = e / ncol;
    const int s = cj / cq, j = cj - s * cq;
    SpreadPiece p;
    p.s = s;
    p.c = c;
    p.j = j;
    p.cl = s * ncol + c;
    p.c1 = c >> 2;
    p.c2 = c & 3;
    return p;
}

// Pair j of column c in a chunk's partial tile, [j][c].
SDP_MAP constexpr int spread_partial_pair(int j, int c, int ncol) { return j * ncol + c; }

// ---------------- forward interpolation (interp_impl.cuh, interp_tiles.cu) ----------------
// Row kernel: lane l of a channel group of cg <= 32 / W channels from c0 owns the
// axis-3 tap a3 = l / cg and channel c0 + l % cg.  Lanes with a3 >= W are idle;
// they repeat the last active lane's tap and channel (with a zero coefficient), so
// their loads stay inside the window.
struct RowLane {
    int a3c;
    int kk;
    bool act;
};

SDP_MAP RowLane row_lane_map(int lane, int c0, int cg, int W) {
    const int a3 = lane / cg, kg = lane - a3 * cg;
    RowLane r;
    r.act = a3 < W;
    r.a3c = r.act ? a3 : W - 1;
    r.kk = c0 + (r.act ? kg : cg - 1);
    return r;
}

// Tiled kernel: lane l16 (< 16) of a half-warp owns the axis-2/axis-3 tap pair
// (a2, a3) = (l16 / W, l16 % W) for l16 < W^2; idle lanes repeat tap (0, 0) with a
// zero weight.
struct TileLane {
    int a2, a3;
    bool act;
};

SDP_MAP TileLane tile_lane_map(int l16, int W) {
    const bool act = l16 < W * W;
    return {act ? l16 / W : 0, act ? l16 % W : 0, act};
}

// Shared-tile offset (in complex values) of tap (a1, a2, a3), channel k, of a sample
// whose window starts at (e1, e2, e3) within a tile of H^3 points x nk channels.
SDP_MAP constexpr int tile_offset(int e1, int e2, int e3, int a1, int a2, int a3, int k, int H, int nk) {
    return ((e1 + a1) * H + e2 + a2) * H * nk + (e3 + a3) * nk + k;
}

// ---------------- fused axis-3 kernels (fft2_impl.cuh, fft2_staged.cu, fft.cu) ----------------
// The grid lines of one coil are l = row nk + kk (channel fastest); FFT position p
// of line l is element (row L + p) nk + kk of the channel-interleaved grid, so the
// positions p + s d of a line are s d nk elements apart.
struct LineRowChannel {
    long long row;
    int kk;
};

SDP_MAP LineRowChannel line_split(long long gl, int nk) {
    const long long row = gl / nk;
    return {row, (int)(gl - row * nk)};
}

// The same split for a line index within a unit of whole rows (32-bit).
struct UnitLine {
    int rr, kk;
};

SDP_MAP UnitLine unit_line_split(int l, int nk) {
    const int rr = l / nk;
    return {rr, l - rr * nk};
}

SDP_MAP long long line_elem(long long row, int L, int p, int nk, int kk) {
    return (row * L + p) * nk + kk;
}

// A thread's (line, position) role in a pass over nl lines: line fastest (the direct
// prologue's pass 2, the direct and staged epilogues' pass 1), or position fastest
// (npos positions a line: the direct prologue's pass 1, the direct and staged
// epilogues' pass 2).
struct LinePos {
    int l, p;
};

SDP_MAP LinePos line_fastest(int tid, int nl) {
    const int p = tid / nl;
    return {tid - p * nl, p};
}

SDP_MAP LinePos pos_fastest(int tid, int npos) { return {tid / npos, tid % npos}; }

// Staged prologue pass 1: thread = (unit line l = rr nk + kk, FFT position b < B), b
// fastest; the thread reads positions B a + b of row rr, channel kk, from shared memory.
struct StagedLoad {
    int l, rr, kk, b;
};

SDP_MAP StagedLoad staged_load_role(int tid, int B, int nk) {
    const int l = tid / B, b = tid - l * B;
    const int rr = l / nk;
    return {l, rr, l - rr * nk, b};
}

// Staged prologue pass 2: thread = (row rr of the unit, FFT index q1 < A, channel kk),
// channel fastest, so for a fixed q2 a warp stores consecutive elements.
struct StagedStore {
    int rr, q1, kk;
};

SDP_MAP StagedStore staged_store_role(int tid, int A, int nk) {
    return {tid / (nk * A), (tid / nk) % A, tid % nk};
}

// Stockham kernels' staged loops: element e of an NL-line block is position p = e / NL
// of block line l = e % NL.
SDP_MAP LinePos stockham_elem(int e, int nl) {
    const int p = e / nl;
    return {e - p * nl, p};
}

}  // namespace imap
}  // namespace sdp
