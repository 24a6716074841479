"""Index arithmetic of the channel-interleaved kernels, checked on the CPU.

The GPU parity tests check results; these check the index maps themselves over
many shapes, so that an edit can be read against them before it runs on a
GPU: every element is written (or read) exactly once, every index stays in its
buffer, and the spread's 16-byte shared-memory writes of a quarter-warp meet
distinct banks.  The maps are the kernels' own: csrc/index_map.cuh, compiled
here for the host (tests/index_map_shim.cpp) and called through ctypes.  The
loops around a map (the lanes of a warp, a thread's FFT positions at a fixed
stride) follow the kernels: spread_impl.cuh (spread_body, store_cols),
interp_impl.cuh (row_lane), interp_tiles.cu (tile_work), fft2_impl.cuh
(fft2_prologue_body, fft2_epilogue_body), fft2_staged.cu and fft.cu.  Nothing
here is method arithmetic; nothing runs on a GPU.
"""
import ctypes
import itertools
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2408_02367_gb300", "csrc")

c_int, c_ll = ctypes.c_int, ctypes.c_longlong


@pytest.fixture(scope="module")
def im(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    lib = tmp_path_factory.mktemp("imap") / "libimap.so"
    r = subprocess.run([cxx, "-std=c++17", "-O1", "-shared", "-fPIC", "-I", CSRC,
                        os.path.join(ROOT, "tests", "index_map_shim.cpp"), "-o", str(lib)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return Maps(ctypes.CDLL(str(lib)))


class Maps:
    """The shim's entry points as Python calls returning tuples."""

    def __init__(self, so):
        self.so = so
        for name, res in (("imap_spread_cq", c_int), ("imap_spread_ts", c_int), ("imap_spread_owns_pair", c_int),
                          ("imap_spread_partial_pair", c_int), ("imap_tile_offset", c_int),
                          ("imap_line_elem", c_ll)):
            getattr(so, name).restype = res
        so.imap_line_elem.argtypes = [c_ll, c_int, c_int, c_int, c_int]
        so.imap_line_split.argtypes = [c_ll, c_int, ctypes.POINTER(c_ll), ctypes.POINTER(c_int)]

    def _rows(self, fn, n, width, *args):
        buf = (c_int * max(1, n * width))()
        fn(n, *args, buf)
        return [tuple(buf[width * e:width * e + width]) for e in range(n)]

    def cq(self, B3, nk):
        return self.so.imap_spread_cq(B3, nk)

    def ts(self, B3, nk):
        return self.so.imap_spread_ts(B3, nk)

    def owns(self, j, ipw, h):
        return bool(self.so.imap_spread_owns_pair(j, ipw, h))

    def partial(self, j, c, ncol):
        return self.so.imap_spread_partial_pair(j, c, ncol)

    def pair_pieces(self, n, cq, ncol):     # (cl, s, c, c1, c2, j)
        return self._rows(self.so.imap_spread_pair_pieces, n, 6, cq, ncol)

    def sum_pieces(self, n, cq, ncol):      # (cl, s, c, c1, c2, j)
        return self._rows(self.so.imap_spread_sum_pieces, n, 6, cq, ncol)

    def value_pieces(self, n, per, nkt, ncol):   # (cl, s, c1, c2, x3, q, r)
        return self._rows(self.so.imap_spread_value_pieces, n, 7, per, nkt, ncol)

    def row_lanes(self, c0, cg, W):         # 32 x (a3c, kk, act)
        buf = (c_int * 96)()
        self.so.imap_row_lanes(c0, cg, W, buf)
        return [tuple(buf[3 * l:3 * l + 3]) for l in range(32)]

    def tile_lanes(self, W):                # 16 x (a2, a3, act)
        buf = (c_int * 48)()
        self.so.imap_tile_lanes(W, buf)
        return [tuple(buf[3 * l:3 * l + 3]) for l in range(16)]

    def tile_offset(self, e, a, k, H, nk):
        return self.so.imap_tile_offset(*e, *a, k, H, nk)

    def line_split(self, gl, nk):
        row, kk = c_ll(), c_int()
        self.so.imap_line_split(gl, nk, ctypes.byref(row), ctypes.byref(kk))
        return row.value, kk.value

    def unit_line_split(self, l, nk):
        rr, kk = c_int(), c_int()
        self.so.imap_unit_line_split(l, nk, ctypes.byref(rr), ctypes.byref(kk))
        return rr.value, kk.value

    def line_elem(self, row, L, p, nk, kk):
        return self.so.imap_line_elem(row, L, p, nk, kk)

    def _lp(self, fn, a, b):
        l, p = c_int(), c_int()
        fn(a, b, ctypes.byref(l), ctypes.byref(p))
        return l.value, p.value

    def line_fastest(self, tid, nl):        # (line, position)
        return self._lp(self.so.imap_line_fastest, tid, nl)

    def pos_fastest(self, tid, npos):       # (line, position)
        return self._lp(self.so.imap_pos_fastest, tid, npos)

    def stockham_elem(self, e, nl):         # (line, position)
        return self._lp(self.so.imap_stockham_elem, e, nl)

    def staged_load_role(self, tid, B, nk):  # (l, rr, kk, b)
        buf = (c_int * 4)()
        self.so.imap_staged_load_role(tid, B, nk, buf)
        return tuple(buf)

    def staged_store_role(self, tid, A, nk):  # (rr, q1, kk)
        buf = (c_int * 3)()
        self.so.imap_staged_store_role(tid, A, nk, buf)
        return tuple(buf)


# ---------------- adjoint spread ----------------

SPREAD_SHAPES = [(B1, B3, NK, NC) for B1 in (8, 4) for B3 in (4, 8) for NK in range(1, 9) for NC in (1, 2)]


def _spread_consts(im, B1, B3, NK, NC):
    NCOL = 4 * B1
    CQ, TS = im.cq(B3, NK), im.ts(B3, NK)
    assert CQ == B3 * NK // 2 and TS % 2 == 1 and CQ <= TS <= CQ + 1
    return NCOL, 32 // NCOL, CQ, TS, max(NC * NCOL, 32)


def _transposition_slots(im, B1, B3, NK, NC):
    """Slots the lanes write when moving their columns' registers to shared memory:
    lane (h, col) writes pair j of coil c at (c NCOL + col) TS + j if it owns j."""
    NCOL, IPW, CQ, TS, _ = _spread_consts(im, B1, B3, NK, NC)
    written = {}
    for lane in range(32):
        h, col = divmod(lane, NCOL)
        for c in range(NC):
            for j in range(CQ):
                if im.owns(j, IPW, h):
                    slot = (c * NCOL + col) * TS + j
                    written[slot] = written.get(slot, 0) + 1
    return written


@pytest.mark.parametrize("B1,B3,NK,NC", SPREAD_SHAPES)
def test_spread_transposition_writes_each_slot_once(im, B1, B3, NK, NC):
    NCOL, IPW, CQ, TS, kTrCols = _spread_consts(im, B1, B3, NK, NC)
    written = _transposition_slots(im, B1, B3, NK, NC)
    expect = {(c * NCOL + col) * TS + j for c in range(NC) for col in range(NCOL) for j in range(CQ)}
    assert set(written) == expect and all(v == 1 for v in written.values())
    assert max(written) < kTrCols * TS


@pytest.mark.parametrize("B1,B3,NK,NC", SPREAD_SHAPES)
def test_spread_bin_store_covers_each_value_once(im, B1, B3, NK, NC):
    """store_cols with the call's full channel set: piece e (lanes take e = lane,
    lane + 32, ...) moves 16-byte pair j of column slot cl from tr[cl TS + j] to
    values 2j, 2j + 1 of column (c1, c2) of coil slot s, when the column lies in the
    grid (c1 < n1, c2 < n2) and the pair below x3end (even: M3 and the bin origin are)."""
    NCOL, IPW, CQ, TS, kTrCols = _spread_consts(im, B1, B3, NK, NC)
    written_slots = set(_transposition_slots(im, B1, B3, NK, NC))
    for nc in range(1, NC + 1):
        pieces = im.pair_pieces(nc * NCOL * CQ, CQ, NCOL)
        for n1, n2, x3end in itertools.product((B1, B1 - 1, 1), (4, 3, 1), range(2, B3 + 1, 2)):
            got = {}
            for cl, s, c, c1, c2, j in pieces:
                assert cl == s * NCOL + c and (c1, c2) == divmod(c, 4) and s < nc
                if c1 < n1 and c2 < n2 and 2 * j < x3end * NK:
                    assert cl * TS + j in written_slots
                    assert 2 * j + 1 < x3end * NK               # a pair never straddles x3end
                    for v in (2 * j, 2 * j + 1):
                        got[(s, c1, c2, v)] = got.get((s, c1, c2, v), 0) + 1
            expect = {(s, c1, c2, v) for s in range(nc) for c1 in range(min(n1, B1)) for c2 in range(min(n2, 4))
                      for v in range(x3end * NK)}
            assert set(got) == expect and all(v == 1 for v in got.values())


@pytest.mark.parametrize("B1,B3,NK,nk", [(8, 4, 5, 10), (8, 8, 4, 9), (4, 4, 5, 16), (4, 8, 3, 7), (4, 4, 1, 3)])
def test_spread_channel_group_store_covers_each_value_once(im, B1, B3, NK, nk):
    """store_cols for a group of NK of the grid's nk channels: 8-byte value
    r = x3 NK + q of column slot cl, read from t2[2 cl TS + r] (pair r / 2, half r % 2)."""
    NCOL, IPW, CQ, TS, kTrCols = _spread_consts(im, B1, B3, NK, 1)
    PER = B3 * NK
    pieces = im.value_pieces(NCOL * PER, PER, NK, NCOL)
    for n1, n2, x3end in itertools.product((B1, 2), (4, 1), range(1, B3 + 1)):
        got = {}
        for cl, s, c1, c2, x3, q, r in pieces:
            assert s == 0 and r == x3 * NK + q and 0 <= r < PER and divmod(2 * cl * TS + r, 2) == (cl * TS + r // 2,
                                                                                              r % 2)
            if c1 < n1 and c2 < n2 and x3 < x3end:
                got[(c1, c2, x3, q)] = got.get((c1, c2, x3, q), 0) + 1
        expect = {(c1, c2, x3, q) for c1 in range(min(n1, B1)) for c2 in range(min(n2, 4)) for x3 in range(x3end)
                  for q in range(NK)}
        assert set(got) == expect and all(v == 1 for v in got.values())


@pytest.mark.parametrize("B1,B3,NK", [(8, 4, 5), (8, 8, 5), (4, 4, 5), (4, 8, 8), (4, 4, 1), (8, 8, 3)])
def test_spread_transposition_buffer_is_conflict_free(im, B1, B3, NK):
    """The transposition's 16-byte writes: for a fixed pair j, the writing lanes of a
    quarter-warp (8 lanes, 128 bytes) hit 8 distinct 16-byte bank groups because TS
    is odd.  The store's reads of the same buffer meet at most two slots per bank
    group (a column boundary skips the pad slot)."""
    NCOL, IPW, CQ, TS, _ = _spread_consts(im, B1, B3, NK, 1)
    for j in range(CQ):
        for q in range(4):
            lanes = [l for l in range(8 * q, 8 * q + 8) if im.owns(j, IPW, l // NCOL)]
            groups = [((l % NCOL) * TS + j) % 8 for l in lanes]
            assert len(set(groups)) == len(groups)
    pieces = im.pair_pieces(NCOL * CQ, CQ, NCOL)
    for base in range(0, len(pieces), 8):
        groups = [(cl * TS + j) % 8 for cl, s, c, c1, c2, j in pieces[base:base + 8]]
        assert max(groups.count(g) for g in set(groups)) <= 2


@pytest.mark.parametrize("B1,B3,NK,NC", SPREAD_SHAPES)
def test_spread_multichunk_partials_and_sum_cover_each_pair_once(im, B1, B3, NK, NC):
    """A chunk's partial tile: lane (h, col) writes pair j of coil c at [j][col] if it
    owns j.  The last chunk's sum: piece e is column c (fastest), pair j, coil slot s;
    it reads [j][c] of every chunk's partial and writes slot (s NCOL + c) TS + j."""
    NCOL, IPW, CQ, TS, kTrCols = _spread_consts(im, B1, B3, NK, NC)
    for c in range(NC):
        got = {}
        for lane in range(32):
            h, col = divmod(lane, NCOL)
            for j in range(CQ):
                if im.owns(j, IPW, h):
                    i = im.partial(j, col, NCOL)
                    got[i] = got.get(i, 0) + 1
        assert set(got) == set(range(CQ * NCOL)) and all(v == 1 for v in got.values())
    per_pass = kTrCols // NCOL
    for npc in range(1, per_pass + 1):
        seen = {}
        for e, (cl, s, c, c1, c2, j) in enumerate(im.sum_pieces(npc * CQ * NCOL, CQ, NCOL)):
            assert c == e % NCOL and cl == s * NCOL + c and (c1, c2) == divmod(c, 4)
            assert j * NCOL + c == im.partial(j, c, NCOL) < CQ * NCOL   # the kernel's read index
            assert cl * TS + j < kTrCols * TS
            seen[(s, c, j)] = seen.get((s, c, j), 0) + 1
        assert set(seen) == {(s, c, j) for s in range(npc) for c in range(NCOL) for j in range(CQ)}
        assert all(v == 1 for v in seen.values())


# ---------------- forward interpolation ----------------

@pytest.mark.parametrize("W", range(2, 9))
@pytest.mark.parametrize("nk", [1, 2, 3, 4, 5, 7, 8, 10, 16])
def test_interp_lanes_cover_taps_and_channels_once(im, W, nk):
    group = 32 // W
    seen = {}
    for c0 in range(0, nk, group):
        cg = min(group, nk - c0)
        for lane, (a3c, kk, act) in enumerate(im.row_lanes(c0, cg, W)):
            assert 0 <= a3c < W and c0 <= kk < c0 + cg <= nk
            if act:
                assert lane < W * cg
                seen[(a3c, kk)] = seen.get((a3c, kk), 0) + 1
            else:
                assert lane >= W * cg
    assert set(seen) == {(a, k) for a in range(W) for k in range(nk)}
    assert all(v == 1 for v in seen.values())


@pytest.mark.parametrize("W", [2, 4])
@pytest.mark.parametrize("nk", [1, 5, 8])
def test_tiled_interp_lanes_and_tile_offsets(im, W, nk):
    """A half-warp's active lanes own each (a2, a3) tap pair once (idle lanes repeat
    (0, 0)); every tap of a window starting at e in [0, 8] per axis lies in the
    (8 + W)^3 x nk tile, and the kernel's offsets a1 H^2 nk + k from its lane's base
    are the map's."""
    lanes = im.tile_lanes(W)
    act = [(a2, a3) for a2, a3, a in lanes if a]
    assert sorted(act) == [(a2, a3) for a2 in range(W) for a3 in range(W)]
    assert all((a2, a3) == (0, 0) for a2, a3, a in lanes if not a)
    H = 8 + W
    size = H ** 3 * nk
    for e in itertools.product((0, 1, 7, 8), repeat=3):
        for a2, a3 in act:
            base = im.tile_offset(e, (0, a2, a3), 0, H, nk)
            for a1 in range(W):
                for k in range(nk):
                    off = im.tile_offset(e, (a1, a2, a3), k, H, nk)
                    assert 0 <= off < size and off == base + a1 * H * H * nk + k


# ---------------- fused axis-3 FFT kernels ----------------

def _count(hits, idx):
    hits[idx] = hits.get(idx, 0) + 1


@pytest.mark.parametrize("A,B,NLT", [(16, 10, 8), (16, 10, 16), (16, 10, 4), (8, 6, 8), (25, 10, 8), (16, 16, 8)])
@pytest.mark.parametrize("nk", [1, 3, 5, 8])
def test_direct_prologue_roles_and_stores_cover_the_lines_once(im, A, B, NLT, nk):
    """fft2_prologue_body: pass-1 thread (line, b) = pos_fastest(tid, B); pass-2 thread
    (l2, q1) = line_fastest(tid, NLT) stores outputs q1 + A q2 at line_elem(row, L, q1,
    nk, kk) + q2 A nk."""
    L = A * B
    nrows = 7                                      # a ragged last line block
    nlines = nrows * nk
    roles = {im.pos_fastest(tid, B) for tid in range(NLT * B)}
    assert roles == {(l, b) for l in range(NLT) for b in range(B)}
    hits = {}
    for l0 in range(0, nlines, NLT):
        for tid in range(NLT * A):
            l2, q1 = im.line_fastest(tid, NLT)
            assert l2 < NLT and q1 < A
            gl = l0 + l2
            if gl >= nlines:
                continue
            row, kk = im.line_split(gl, nk)
            assert row * nk + kk == gl and 0 <= kk < nk
            d0 = im.line_elem(row, L, q1, nk, kk)
            for q2 in range(B):
                idx = d0 + q2 * A * nk
                assert idx == im.line_elem(row, L, q1 + A * q2, nk, kk) and 0 <= idx < nrows * L * nk
                _count(hits, idx)
    assert len(hits) == nrows * L * nk and all(v == 1 for v in hits.values())


@pytest.mark.parametrize("A,B,NLT", [(16, 10, 8), (16, 10, 16), (16, 10, 4), (8, 6, 8), (25, 10, 8)])
@pytest.mark.parametrize("nk", [1, 2, 5, 8])
def test_direct_epilogue_roles_and_loads_cover_the_lines_once(im, A, B, NLT, nk):
    """fft2_epilogue_body: pass-1 thread (l1, b1) = line_fastest(tid, NLT) loads FFT
    positions B a + b1 from line_elem(row, L, b1, nk, kk) in steps of B nk; pass-2
    thread (l2, q1) = pos_fastest(tid, A)."""
    L = A * B
    nrows = 6
    nlines = nrows * nk
    hits = {}
    for l0 in range(0, nlines, NLT):
        for tid in range(NLT * B):
            l1, b1 = im.line_fastest(tid, NLT)
            gl = l0 + l1
            if gl >= nlines:
                continue
            row, kk = im.line_split(gl, nk)
            idx = im.line_elem(row, L, b1, nk, kk)
            for a in range(A):
                assert 0 <= idx < nrows * L * nk and (idx - kk) // nk % B == b1
                _count(hits, idx)
                idx += B * nk
    assert len(hits) == nrows * L * nk and all(v == 1 for v in hits.values())
    roles = {im.pos_fastest(tid, A) for tid in range(NLT * A)}
    assert roles == {(l, q) for l in range(NLT) for q in range(A)}


@pytest.mark.parametrize("A,B", [(16, 10), (20, 10), (25, 10), (8, 6), (16, 16)])
@pytest.mark.parametrize("nk", [1, 3, 5, 8])
def test_staged_prologue_roles_and_stores_cover_the_unit_once(im, A, B, nk):
    """fft2_staged.cu prologue, a unit of R rows (NL = R nk lines): pass-1 thread
    staged_load_role(tid, B, nk) = (l, rr, kk, b); pass-2 thread staged_store_role(tid,
    A, nk) = (rr, q1, kk) stores q1 + A q2 at line_elem(row0 + rr, L, q1, nk, kk) +
    q2 A nk, consecutive threads of a row writing consecutive elements."""
    threads = 512 if A * B >= 200 else 256
    R = threads // max(A, B) // nk
    if R < 1:
        pytest.skip("a row's channels do not fit a unit")
    NL, L = R * nk, A * B
    seen = set()
    for tid in range(NL * B):
        l, rr, kk, b = im.staged_load_role(tid, B, nk)
        assert l == rr * nk + kk and rr < R and kk < nk and b < B
        seen.add((rr, kk, b))
    assert len(seen) == NL * B
    row0 = 3
    hits = {}
    prev = None
    for tid in range(NL * A):
        rr, q1, kk = im.staged_store_role(tid, A, nk)
        assert rr < R and q1 < A and kk < nk
        d0 = im.line_elem(row0 + rr, L, q1, nk, kk)
        if prev is not None and prev[0] == rr:
            assert d0 == prev[1] + 1                  # a warp's stores of one q2 are contiguous
        prev = (rr, d0)
        for q2 in range(B):
            _count(hits, d0 + q2 * A * nk)
    lo = row0 * L * nk
    assert set(hits) == set(range(lo, lo + R * L * nk)) and all(v == 1 for v in hits.values())


@pytest.mark.parametrize("A,B", [(16, 10), (20, 10), (25, 10), (8, 6), (16, 16)])
@pytest.mark.parametrize("nk", [1, 3, 5, 8])
def test_staged_epilogue_roles_and_loads_cover_the_unit_once(im, A, B, nk):
    """fft2_staged.cu epilogue: pass-1 thread (l1, b1) = line_fastest(tid, NL), (rr, kk)
    = unit_line_split(l1, nk), loads gs[line_elem(rr, L, B a + b1, nk, kk)] of the
    staged [rr][L][nk] lines; pass-2 thread (l2, q1) = pos_fastest(tid, A)."""
    threads = 512 if A * B >= 200 else 256
    R = threads // max(A, B) // nk
    if R < 1:
        pytest.skip("a row's channels do not fit a unit")
    NL, L = R * nk, A * B
    hits = {}
    for tid in range(NL * B):
        l1, b1 = im.line_fastest(tid, NL)
        rr, kk = im.unit_line_split(l1, nk)
        assert rr * nk + kk == l1 and rr < R
        for a in range(A):
            _count(hits, im.line_elem(rr, L, B * a + b1, nk, kk))
    assert set(hits) == set(range(R * L * nk)) and all(v == 1 for v in hits.values())
    roles = set()
    for tid in range(NL * A):
        l2, q1 = im.pos_fastest(tid, A)
        rr, kk = im.unit_line_split(l2, nk)
        assert rr < R and q1 < A
        roles.add((rr, kk, q1))
    assert len(roles) == NL * A


@pytest.mark.parametrize("L", [48, 81, 150, 160])
@pytest.mark.parametrize("nk", [1, 5, 16])
def test_stockham_axis3_interleaved_loops_cover_the_lines_once(im, L, nk):
    """Store loop of the Stockham forward prologue and load loop of its adjoint
    epilogue: element e of a block is (line, position) = stockham_elem(e, NL) at
    line_elem(row, L, p, nk, kk)."""
    NL, threads = 16, 256
    nrows = 5
    nlines = nrows * nk
    hits = {}
    for l0 in range(0, nlines, NL):
        for t in range(threads):
            for e in range(t, NL * L, threads):
                l, p = im.stockham_elem(e, NL)
                assert l < NL and p < L
                gl = l0 + l
                if gl >= nlines:
                    continue
                row, kk = im.line_split(gl, nk)
                idx = im.line_elem(row, L, p, nk, kk)
                assert 0 <= idx < nrows * L * nk
                _count(hits, idx)
    assert len(hits) == nrows * L * nk and all(v == 1 for v in hits.values())
