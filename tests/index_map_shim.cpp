// Host build of the kernels' index maps (paper_2408_02367_gb300/csrc/index_map.cuh)
// for the CPU tests in test_index_math.py.  Each entry point evaluates one map of
// the header for the arguments given (the enumerating ones over e = 0 .. n - 1)
// and writes the fields into caller-provided arrays, so the tests check the
// arithmetic the kernels compile, not a restatement of it.  Compiled by the
// tests with the host C++ compiler; nothing here runs on a GPU.
#include "index_map.cuh"

using namespace sdp::imap;

extern "C" {

int imap_spread_cq(int B3, int nk) { return spread_cq(B3, nk); }
int imap_spread_ts(int B3, int nk) { return spread_ts(B3, nk); }
int imap_spread_owns_pair(int j, int ipw, int h) { return spread_owns_pair(j, ipw, h) ? 1 : 0; }
int imap_spread_partial_pair(int j, int c, int ncol) { return spread_partial_pair(j, c, ncol); }

// out[6 e ..] = cl, s, c, c1, c2, j
void imap_spread_pair_pieces(int n, int cq, int ncol, int* out) {
    for (int e = 0; e < n; ++e) {
        const SpreadPiece p = spread_pair_piece(e, cq, ncol);
        const int v[6] = {p.cl, p.s, p.c, p.c1, p.c2, p.j};
        for (int f = 0; f < 6; ++f) out[6 * e + f] = v[f];
    }
}

void imap_spread_sum_pieces(int n, int cq, int ncol, int* out) {
    for (int e = 0; e < n; ++e) {
        const SpreadPiece p = spread_sum_piece(e, cq, ncol);
        const int v[6] = {p.cl, p.s, p.c, p.c1, p.c2, p.j};
        for (int f = 0; f < 6; ++f) out[6 * e + f] = v[f];
    }
}

// out[7 e ..] = cl, s, c1, c2, x3, q, r
void imap_spread_value_pieces(int n, int per, int nkt, int ncol, int* out) {
    for (int e = 0; e < n; ++e) {
        const SpreadValue p = spread_value_piece(e, per, nkt, ncol);
        const int v[7] = {p.cl, p.s, p.c1, p.c2, p.x3, p.q, p.r};
        for (int f = 0; f < 7; ++f) out[7 * e + f] = v[f];
    }
}

// out[3 lane ..] = a3c, kk, act for the 32 lanes
void imap_row_lanes(int c0, int cg, int W, int* out) {
    for (int lane = 0; lane < 32; ++lane) {
        const RowLane r = row_lane_map(lane, c0, cg, W);
        out[3 * lane] = r.a3c;
        out[3 * lane + 1] = r.kk;
        out[3 * lane + 2] = r.act ? 1 : 0;
    }
}

// out[3 l16 ..] = a2, a3, act for the 16 lanes of a half-warp
void imap_tile_lanes(int W, int* out) {
    for (int l = 0; l < 16; ++l) {
        const TileLane t = tile_lane_map(l, W);
        out[3 * l] = t.a2;
        out[3 * l + 1] = t.a3;
        out[3 * l + 2] = t.act ? 1 : 0;
    }
}

int imap_tile_offset(int e1, int e2, int e3, int a1, int a2, int a3, int k, int H, int nk) {
    return tile_offset(e1, e2, e3, a1, a2, a3, k, H, nk);
}

void imap_line_split(long long gl, int nk, long long* row, int* kk) {
    const LineRowChannel r = line_split(gl, nk);
    *row = r.row;
    *kk = r.kk;
}

void imap_unit_line_split(int l, int nk, int* rr, int* kk) {
    const UnitLine u = unit_line_split(l, nk);
    *rr = u.rr;
    *kk = u.kk;
}

long long imap_line_elem(long long row, int L, int p, int nk, int kk) { return line_elem(row, L, p, nk, kk); }

void imap_line_fastest(int tid, int nl, int* l, int* p) {
    const LinePos r = line_fastest(tid, nl);
    *l = r.l;
    *p = r.p;
}

void imap_pos_fastest(int tid, int npos, int* l, int* p) {
    const LinePos r = pos_fastest(tid, npos);
    *l = r.l;
    *p = r.p;
}

void imap_stockham_elem(int e, int nl, int* l, int* p) {
    const LinePos r = stockham_elem(e, nl);
    *l = r.l;
    *p = r.p;
}

// out[4] = l, rr, kk, b
void imap_staged_load_role(int tid, int B, int nk, int* out) {
    const StagedLoad s = staged_load_role(tid, B, nk);
    out[0] = s.l;
    out[1] = s.rr;
    out[2] = s.kk;
    out[3] = s.b;
}

// out[3] = rr, q1, kk
void imap_staged_store_role(int tid, int A, int nk, int* out) {
    const StagedStore s = staged_store_role(tid, A, nk);
    out[0] = s.rr;
    out[1] = s.q1;
    out[2] = s.kk;
}

}  // extern "C"
