"""Planted mistakes in the oracle must be caught by the pins.

Each case copies the oracle's source, plants one plausible mistake (a dropped
term, a wrong sign or index, a transposed operand), loads the copy as a separate
module and runs the pins of tests/oracle_pins.py against it.  At least one pin
must fail for every planted mistake.  CPU only; the real oracle is untouched.
"""
import importlib.util
import os
import types

import pytest

from tests import oracle_pins as P

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "nufft.py")

MUTATIONS = {
    "deapod_sin_branch_as_sinh": ("neg = np.sin(z) / z", "neg = np.sinh(z) / z"),
    "deapod_missing_i0_norm": ("return W * val / np.i0(beta)", "return W * val"),
    "window_without_norm": ("return np.i0(beta * np.sqrt(np.maximum(t, 0.0))) / np.i0(beta)\n\n\n#",
                            "return np.i0(beta * np.sqrt(np.maximum(t, 0.0)))\n\n\n#"),
    "nudft_forward_sign": ("_phase_factors(omega[j0:j1], n, -1.0)", "_phase_factors(omega[j0:j1], n, +1.0)"),
    "centring_off_by_one": ("return np.arange(nd) - nd // 2", "return np.arange(nd) - nd // 2 + 1"),
    "nudft_adjoint_no_conj_V": ("w = np.conj(V[frame[j0:j1]]) * y[b, j0:j1, None]",
                                "w = V[frame[j0:j1]] * y[b, j0:j1, None]"),
    "nudft_adjoint_no_conj_S": ("out += np.conj(S[c])[None] * h", "out += S[c][None] * h"),
    "spread_no_conj_V": ("c = np.conj(V[frame[j0:j1], k]) * r[j0:j1]", "c = V[frame[j0:j1], k] * r[j0:j1]"),
    "interp_V_transposed": ("y[j0:j1] = np.sum(_as_c128(V)[frame[j0:j1]] * acc, axis=1)",
                            "y[j0:j1] = np.sum((_as_c128(V).T if V.shape[0] == V.shape[1] else _as_c128(V))[frame[j0:j1]] * acc, axis=1)"),
    "deapod_multiplied": ("u = _as_c128(S_c) * _as_c128(x_k) / geo.psi_hat()",
                          "u = _as_c128(S_c) * _as_c128(x_k) * geo.psi_hat()"),
    "epilogue_deapod_missing": ("return np.conj(_as_c128(S_c)) * crop / geo.psi_hat()",
                                "return np.conj(_as_c128(S_c)) * crop"),
    "window_start_floor": ("return np.ceil(g32 - np.float32(W / 2.0)).astype(np.int64)",
                           "return np.floor(g32 - np.float32(W / 2.0)).astype(np.int64)"),
    "coil_map_dropped": ("u = _as_c128(S_c) * _as_c128(x_k) / geo.psi_hat()",
                         "u = _as_c128(x_k) / geo.psi_hat()"),
    "ifft_normalised": ("return np.fft.ifftn(H) * H.size", "return np.fft.ifftn(H)"),
    "grid_coord_sign": ("g = om[:, d] * s", "g = -om[:, d] * s"),
    "tap_axes_swapped": ("flat = (i1[:, :, None, None] * M[1] + i2[:, None, :, None]) * M[2] + i3[:, None, None, :]",
                         "flat = (i1[:, :, None, None] * M[1] + i3[:, None, None, :]) * M[2] + i2[:, None, :, None]"),
    "tap_weight_axes_mixed": ("return (w[:, 0, :, None, None] * w[:, 1, None, :, None] * w[:, 2, None, None, :])",
                              "return (w[:, 0, :, None, None] * w[:, 0, None, :, None] * w[:, 2, None, None, :])"),
    "beta_wrong_half": ("(sigma - 0.5) ** 2 - 0.8", "(sigma - 0.25) ** 2 - 0.8"),
}


def _load_mutant(old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique/found: {old!r}"
    mod = types.ModuleType("oracle_mutant")
    exec(compile(src.replace(old, new), "oracle_mutant", "exec"), mod.__dict__)
    return mod


def _pins_fail(O):
    """Run the pins; return the names of those that fail (an exception counts as failing)."""
    checks = {
        "kb_ft": lambda: P.kb_ft_vs_quadrature(O) < 1e-10,
        "nudft_fftn": lambda: P.nudft_on_grid_vs_fftn(O) < 1e-12,
        "gram": lambda: P.full_cartesian_gram(O) < 1e-12,
        "grid_fwd": lambda: P.gridding_vs_nudft(O, 6, 2.0, n=(10, 12, 8), J=150) < 2e-5,
        "grid_adj": lambda: P.gridding_vs_nudft(O, 6, 2.0, n=(10, 12, 8), J=150, adjoint=True) < 2e-5,
        "perm_V": lambda: P.subspace_permutation(O) < 2e-5,
        "adj_ident": lambda: P.adjoint_identity(O, n=(10, 8, 12), J=200) < 1e-12,
    }
    failed = []
    for name, fn in checks.items():
        try:
            ok = bool(fn())
        except Exception:
            ok = False
        if not ok:
            failed.append(name)
    return failed


def test_unmutated_copy_passes_every_pin():
    assert _pins_fail(_load_mutant("TWO_PI = 2.0 * np.pi", "TWO_PI = 2.0 * np.pi")) == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name):
    old, new = MUTATIONS[name]
    failed = _pins_fail(_load_mutant(old, new))
    print(name, "caught by", failed)
    assert failed, f"planted mistake {name} passed every pin"
