"""Pins of the dictionary-matching oracle (CPU only).

Each pin comes from a fact other than the oracle's own formula: Cauchy-Schwarz
(a voxel that is a scaled atom is matched to that atom, with that scale), the
least-squares characterisation (the matched atom is the best rank-one fit, and
PD is numpy's lstsq coefficient), invariances under scaling and permutation,
and the stated tie and zero readings.  Planted mistakes must fail a pin.
"""
import types

import numpy as np
import pytest

from oracle import dm as DM
from paper_2408_02367_gb300 import synth


@pytest.fixture(scope="module")
def dictionary():
    f, params = synth.mrf_dictionary(120, n_t1=16, n_t2=12)
    D, V = synth.compress_dictionary(f, 5)
    return D.astype(np.complex128), params


def test_planted_atoms_recovered_with_their_scale(dictionary):
    D, _ = dictionary
    x, p, pd = synth.dm_volume(D, 400, noise=0.0, seed=11)
    x = (pd[:, None] * D[p]).T                        # exact in float64
    idx, pd_hat = DM.dictionary_match(x, D)
    assert np.array_equal(idx, p)
    assert np.max(np.abs(pd_hat - pd) / np.abs(pd)) < 1e-10


def test_matched_atom_is_the_best_least_squares_rank_one_fit(dictionary):
    D, _ = dictionary
    rng = np.random.default_rng(12)
    x = rng.standard_normal((5, 60)) + 1j * rng.standard_normal((5, 60))
    idx, pd = DM.dictionary_match(x, D)
    for v in range(x.shape[1]):
        res = []
        for p in range(D.shape[0]):
            c, r, _, _ = np.linalg.lstsq(D[p][:, None], x[:, v], rcond=None)
            res.append(np.linalg.norm(x[:, v] - D[p] * c[0]))
            if p == idx[v]:
                assert abs(c[0] - pd[v]) < 1e-10 * max(1.0, abs(c[0]))
        res = np.array(res)
        assert res[idx[v]] <= res.min() * (1 + 1e-12) + 1e-14


def test_invariances(dictionary):
    D, _ = dictionary
    x, _, _ = synth.dm_volume(D, 200, noise=0.05, seed=13)
    idx, pd = DM.dictionary_match(x, D)
    c = 0.3 - 1.7j
    idx2, pd2 = DM.dictionary_match(c * x.astype(np.complex128), D)
    assert np.array_equal(idx, idx2)
    assert np.allclose(pd2, c * pd, rtol=1e-10, atol=0)
    # scaling atom q by a: same matches, PD of its voxels divided by a
    q = int(idx[0])
    a = 2.5 + 0.5j
    D2 = D.copy()
    D2[q] *= a
    idx3, pd3 = DM.dictionary_match(x, D2)
    assert np.array_equal(idx, idx3)
    sel = idx == q
    assert np.allclose(pd3[sel], pd[sel] / a, rtol=1e-10, atol=0)
    # permuting the atoms permutes the indices
    perm = np.random.default_rng(14).permutation(D.shape[0])
    idx4, pd4 = DM.dictionary_match(x, D[perm])
    assert np.array_equal(perm[idx4], idx)
    assert np.allclose(pd4, pd, rtol=1e-12, atol=0)


def test_ties_zero_voxel_and_zero_atom():
    D = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 0], [0, 2, 0], [1, 1, 0]], np.complex128)
    x = np.array([[0, 0, 1], [3, 0, 1], [0, 0, 0]], np.complex128)  # voxels: e2*3, 0, e1+e2
    idx, pd = DM.dictionary_match(x, D)
    assert idx[0] == 1 and abs(pd[0] - 3) < 1e-15            # atoms 1 and 3 tie: the first wins
    assert idx[1] == 0 and pd[1] == 0                         # zero voxel
    assert idx[2] == 4 and abs(pd[2] - 1) < 1e-15             # |e1+e2| / sqrt2 beats 1 / 1
    assert DM.normalised_scores(x, D)[2].max() == 0           # a zero atom scores 0


MUTATIONS = {
    "no_atom_normalisation": ("score = np.abs(s) * inv[:, None]", "score = np.abs(s)"),
    "real_part_score": ("score = np.abs(s) * inv[:, None]", "score = np.real(s) * inv[:, None]"),
    "pd_single_norm": ("pd[v0:v1] = s[i, cols] * inv[i] ** 2", "pd[v0:v1] = s[i, cols] * inv[i]"),
    "pd_conjugated": ("pd[v0:v1] = s[i, cols] * inv[i] ** 2", "pd[v0:v1] = np.conj(s[i, cols]) * inv[i] ** 2"),
    "no_conj_atoms": ("s = D.conj() @ xv[:, v0:v1]", "s = D @ xv[:, v0:v1]"),
    "argmin": ("i = np.argmax(score, axis=0)", "i = np.argmin(score, axis=0)"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistakes_fail_a_pin(name, dictionary):
    import inspect
    old, new = MUTATIONS[name]
    src = inspect.getsource(DM)
    assert src.count(old) == 1
    mod = types.ModuleType("dm_mutant")
    exec(compile(src.replace(old, new), "dm_mutant", "exec"), mod.__dict__)
    fails = 0
    for pin in (test_planted_atoms_recovered_with_their_scale, test_matched_atom_is_the_best_least_squares_rank_one_fit,
                test_invariances, lambda d: test_ties_zero_voxel_and_zero_atom()):
        saved = DM.dictionary_match, DM.normalised_scores
        try:
            DM.dictionary_match, DM.normalised_scores = mod.dictionary_match, mod.normalised_scores
            pin(dictionary)
        except AssertionError:
            fails += 1
        finally:
            DM.dictionary_match, DM.normalised_scores = saved
    assert fails > 0, name
