"""FP64 oracle of MRF dictionary matching (DM).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the benchmark's
CPU-baseline / reference leg may import this module; the product path never does,
and this module imports nothing from the product package.

What it computes (StoDIP, Sec. 2 after Eq. 1: DM, after Ma et al. 2013 and
McGivney et al. 2014, inverts the voxel-wise Bloch response x_v = PD_v B(T1_v, T2_v)
of the reconstructed TSMI to give the Q-maps).  With the TSMI x_v in C^K of voxel
v and the compressed dictionary atoms d_p in C^K (p = 0..P-1):

    p*(v) = argmax_p |d_p^H x_v| / ||d_p||
    PD_v  = d_{p*}^H x_v / ||d_{p*}||^2

and (T1_v, T2_v) are the parameters of atom p*(v).  This is the least-squares
rank-one fit: for each atom the best complex scale is c_p = d_p^H x_v / ||d_p||^2
with residual ||x_v||^2 - |d_p^H x_v|^2 / ||d_p||^2, so the matched atom is the one
with the smallest residual and PD_v is its scale.

Readings where the paper is silent: PD is kept complex (its magnitude is the usual
PD map); on equal scores the lowest atom index wins; an atom of zero norm scores 0;
a zero voxel is matched to atom 0 with PD 0.
"""
from __future__ import annotations

import numpy as np


def dictionary_match(x, D, chunk: int = 2048):
    """x [K][...] (any trailing voxel shape), D [P][K] -> (idx int64 [nvox], PD complex128 [nvox])."""
    D = np.asarray(D, np.complex128)
    K = D.shape[1]
    xv = np.asarray(x, np.complex128).reshape(K, -1)
    nvox = xv.shape[1]
    nrm = np.linalg.norm(D, axis=1)
    inv = np.where(nrm > 0, 1.0 / np.where(nrm > 0, nrm, 1.0), 0.0)
    idx = np.zeros(nvox, np.int64)
    pd = np.zeros(nvox, np.complex128)
    for v0 in range(0, nvox, chunk):
        v1 = min(nvox, v0 + chunk)
        s = D.conj() @ xv[:, v0:v1]                        # [P][n]: d_p^H x_v
        score = np.abs(s) * inv[:, None]
        i = np.argmax(score, axis=0)                       # first index on ties
        cols = np.arange(v1 - v0)
        idx[v0:v1] = i
        pd[v0:v1] = s[i, cols] * inv[i] ** 2
    return idx, pd


def normalised_scores(x, D):
    """|d_p^H x_v| / ||d_p|| for all atoms and voxels, [P][nvox] (for validity checks)."""
    D = np.asarray(D, np.complex128)
    xv = np.asarray(x, np.complex128).reshape(D.shape[1], -1)
    nrm = np.linalg.norm(D, axis=1)
    inv = np.where(nrm > 0, 1.0 / np.where(nrm > 0, nrm, 1.0), 0.0)
    return np.abs(D.conj() @ xv) * inv[:, None]
