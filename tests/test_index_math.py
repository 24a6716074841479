"""Index arithmetic of the channel-interleaved kernels, checked on the CPU.

The GPU parity tests check results; these check the mappings themselves over
many shapes, so that an edit can be read against them before it runs on a
GPU: every element is written exactly once and every index stays in its
buffer.  The mappings are restated from their definitions in the kernels'
comments (csrc/spread_impl.cuh store_bin, csrc/interp.cu interp_rows_kernel,
csrc/fft2.cu fft2_fwd_prologue_kernel and fft2_adj_epilogue_kernel, csrc/fft.cu
fwd_prologue_fft3_kernel and adj_fft3_epilogue_kernel); nothing here is method
arithmetic.
"""
import itertools

import pytest


def spread_store_targets(B3, NK, n1, n2, x3end):
    """(column, element) pairs the warp stores for one bin, with the shared-memory
    slots they are read from: pair e = r * 32 + lane of column e // CQ."""
    CQ = B3 * NK // 2
    TS = CQ | 1
    out = []
    for r in range(CQ):
        for lane in range(32):
            e = r * 32 + lane
            c, j = divmod(e, CQ)
            c1, c2 = c >> 2, c & 3
            if c1 < n1 and c2 < n2 and 2 * j < x3end * NK:
                out.append(((c1, c2), 2 * j, c * TS + j))
    return out, CQ, TS


@pytest.mark.parametrize("B3", [4, 8])
@pytest.mark.parametrize("NK", range(1, 9))
def test_spread_bin_store_covers_each_value_once(B3, NK):
    for n1, n2, x3end in itertools.product((8, 5, 1), (4, 3, 1), range(2, B3 + 1, 2)):
        targets, CQ, TS = spread_store_targets(B3, NK, n1, n2, x3end)
        written = {}
        for col, e0, slot in targets:
            assert 0 <= slot < 32 * TS
            for e in (e0, e0 + 1):
                x3 = e // NK
                assert x3 < x3end                      # a pair never straddles x3end
                written[(col, e)] = written.get((col, e), 0) + 1
        expect = {((c1, c2), e) for c1 in range(min(n1, 8)) for c2 in range(min(n2, 4))
                  for e in range(x3end * NK)}
        assert set(written) == expect and all(v == 1 for v in written.values())


@pytest.mark.parametrize("B3,NK", [(4, 5), (8, 5), (4, 8), (8, 8), (4, 1), (8, 3)])
def test_spread_transposition_buffer_is_conflict_free(B3, NK):
    """16-byte writes tr[lane * TS + j]: each quarter-warp (8 lanes, 128 bytes) hits
    8 distinct 16-byte bank groups because TS is odd."""
    CQ = B3 * NK // 2
    TS = CQ | 1
    assert TS % 2 == 1
    for j in range(CQ):
        for q in range(4):
            groups = {((8 * q + l) * TS + j) % 8 for l in range(8)}
            assert len(groups) == 8


@pytest.mark.parametrize("W", range(2, 9))
@pytest.mark.parametrize("nk", [1, 2, 3, 4, 5, 7, 8, 10, 16])
def test_interp_lanes_cover_taps_and_channels_once(W, nk):
    group = 32 // W
    seen = {}
    for c0 in range(0, nk, group):
        cg = min(group, nk - c0)
        for lane in range(32):
            a3, kg = divmod(lane, cg)
            act = a3 < W
            a3c = a3 if act else W - 1
            kk = c0 + (kg if act else cg - 1)
            assert 0 <= a3c < W and c0 <= kk < c0 + cg < nk + 1
            if act:
                seen[(a3, kk)] = seen.get((a3, kk), 0) + 1
    assert set(seen) == {(a, k) for a in range(W) for k in range(nk)}
    assert all(v == 1 for v in seen.values())


@pytest.mark.parametrize("A,B,NLT", [(16, 10, 8), (16, 10, 16), (16, 10, 4), (8, 6, 8), (25, 10, 8), (16, 16, 8)])
@pytest.mark.parametrize("nk", [1, 3, 5, 8])
def test_prologue_interleaved_stores_cover_the_lines_once(A, B, NLT, nk):
    """Pass 2 of the fused forward kernel: thread (l2 = tid % NLT, q1 = tid / NLT)
    stores outputs q1 + A q2 of line l0 + l2 at ((row L + q1 + A q2) nk + kk)."""
    L = A * B
    nrows = 7                                      # a ragged last line block
    nlines = nrows * nk
    hits = {}
    for l0 in range(0, nlines, NLT):
        for tid in range(NLT * max(A, B)):
            if tid >= NLT * A:
                continue
            l2, q1 = tid % NLT, tid // NLT
            gl = l0 + l2
            if gl >= nlines:
                continue
            row, kk = divmod(gl, nk)
            for q2 in range(B):
                idx = (row * L + q1 + A * q2) * nk + kk
                assert 0 <= idx < nrows * L * nk
                hits[idx] = hits.get(idx, 0) + 1
    assert len(hits) == nrows * L * nk and all(v == 1 for v in hits.values())


@pytest.mark.parametrize("A,B,NLT", [(16, 10, 8), (16, 10, 16), (16, 10, 4), (8, 6, 8), (25, 10, 8)])
@pytest.mark.parametrize("nk", [1, 2, 5, 8])
def test_epilogue_interleaved_loads_cover_the_lines_once(A, B, NLT, nk):
    """Pass 1 of the fused adjoint kernel: thread (l1 = tid % NLT, b1 = tid / NLT)
    loads FFT positions B a + b1 of line l0 + l1 from a running pointer that
    starts at ((row L + b1) nk + kk) and steps by B nk."""
    L = A * B
    nrows = 6
    nlines = nrows * nk
    hits = {}
    for l0 in range(0, nlines, NLT):
        for tid in range(NLT * max(A, B)):
            if tid >= NLT * B:
                continue
            l1, b1 = tid % NLT, tid // NLT
            gl = l0 + l1
            if gl >= nlines:
                continue
            row, kk = divmod(gl, nk)
            idx = (row * L + b1) * nk + kk
            for a in range(A):
                assert 0 <= idx < nrows * L * nk and (idx - kk) // nk % B == b1
                hits[idx] = hits.get(idx, 0) + 1
                idx += B * nk
    assert len(hits) == nrows * L * nk and all(v == 1 for v in hits.values())


@pytest.mark.parametrize("L", [48, 81, 150, 160])
@pytest.mark.parametrize("nk", [1, 5, 16])
def test_stockham_axis3_interleaved_loops_cover_the_lines_once(L, nk):
    """Store loop of the Stockham forward prologue and load loop of its adjoint
    epilogue: e -> (p = e / NL, l = e % NL), grid index ((row L + p) nk + kk)."""
    NL, threads = 16, 256
    nrows = 5
    nlines = nrows * nk
    hits = {}
    for l0 in range(0, nlines, NL):
        for t in range(threads):
            for e in range(t, NL * L, threads):
                p, l = divmod(e, NL)
                gl = l0 + l
                if gl >= nlines:
                    continue
                row, kk = divmod(gl, nk)
                idx = (row * L + p) * nk + kk
                assert 0 <= idx < nrows * L * nk
                hits[idx] = hits.get(idx, 0) + 1
    assert len(hits) == nrows * L * nk and all(v == 1 for v in hits.values())
