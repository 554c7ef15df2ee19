"""Planted mistakes in the warm-start operator's oracle, each caught by a pin
of tests/test_oracle_fno.py (the mistake is patched in for one test only)."""

import numpy as np
import pytest

import test_oracle_fno as T
from oracle import fno


def _fails(fn, *a):
    with pytest.raises(AssertionError):
        fn(*a)


def test_positive_ky_only_is_caught(monkeypatch):
    monkeypatch.setattr(fno, "KY", np.concatenate([np.arange(16), np.arange(16, 32)]))
    _fails(T.test_identity_weights_give_the_kept_mode_projection)


def test_missing_hermitian_weight_in_backward_is_caught(monkeypatch):
    real_backward = fno.backward

    def bad_mode_ky_kx():
        ky, kx = np.tile(fno.KY, fno.MODES), np.repeat(fno.KX, 2 * fno.MODES)
        return ky, np.zeros_like(kx)        # every mode weighted as kx = 0
    monkeypatch.setattr(fno, "mode_ky_kx", bad_mode_ky_kx)
    _fails(T.test_backward_matches_finite_differences, "spec_w", 3, (33, 5, 7))
    assert fno.backward is real_backward


def test_missing_conjugate_in_weight_gradient_is_caught(monkeypatch):
    real_einsum = np.einsum

    def einsum(sub, *ops, **kw):
        if sub == "bom,bim->moi":
            ops = (ops[0], np.conj(ops[1]))   # undoes the conjugate the oracle applies
        return real_einsum(sub, *ops, **kw)
    monkeypatch.setattr(fno.np, "einsum", einsum)
    _fails(T.test_backward_matches_finite_differences, "spec_w", 3, (33, 5, 7))


def test_gelu_derivative_without_second_term_is_caught(monkeypatch):
    from scipy.special import erf
    monkeypatch.setattr(fno, "gelu_grad", lambda z: 0.5 * (1.0 + erf(z / np.sqrt(2.0))))
    _fails(T.test_backward_matches_finite_differences, "pw_w", 1, (4, 9))
