"""Pins of the warm-start operator's oracle (oracle/fno.py) against facts
that do not come from the oracle's own code:

* the backward pass equals central finite differences of the forward pass
  (float64), for entries of every parameter group, including the complex
  spectral weights' real and imaginary parts;
* the spectral convolution with R_m = identity is the projection onto the
  kept Fourier modes, written here as an explicit double sum of cosines and
  sines over those modes (no FFT);
* a single kept Fourier mode through R_m = r I comes out multiplied by r, a
  mode that is not kept comes out as zero;
* the spectral convolution commutes with circular shifts of the grid;
* bfloat16 rounding: exact values stay, halfway cases go to even, and the
  rounding error is at most 2^-8 relative (half of the 2^-7 spacing).
"""

import numpy as np
import pytest

from oracle import fno
from paper_1102_3069_gb300 import inputs

N = 128
# the kept modes as specified: 16 per axis and sign (kx >= 0 in the half spectrum)
KY_SPEC = list(range(16)) + list(range(N - 16, N))
KX_SPEC = list(range(16))


def _explicit_lowpass(v):
    """sum over kept modes of (w(kx)/N^2) Re(Vhat e^{i theta}), Vhat by a direct sum."""
    y, x = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    out = np.zeros_like(v)
    for ky in KY_SPEC:
        for kx in KX_SPEC:
            th = 2 * np.pi * (ky * y + kx * x) / N
            vh = (v * np.cos(th)).sum(axis=(-2, -1)) - 1j * (v * np.sin(th)).sum(axis=(-2, -1))
            w = 1.0 if kx == 0 else 2.0
            out += (w / N ** 2) * np.real(vh[..., None, None] * np.exp(1j * th))
    return out


def test_identity_weights_give_the_kept_mode_projection():
    g = np.random.default_rng(1)
    v = g.standard_normal((1, 2, N, N))
    R = np.broadcast_to(np.eye(2), (fno.NMODE, 2, 2)).astype(complex)
    S, _, _ = fno.spectral_conv(v, R)
    ref = _explicit_lowpass(v)
    assert np.max(np.abs(S - ref)) < 1e-10 * np.max(np.abs(ref))


def test_single_mode_scaled_and_dropped_modes_removed():
    y, x = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    r = 0.7 - 0.3j
    R = np.broadcast_to(r * np.eye(1), (fno.NMODE, 1, 1)).astype(complex)
    for ky, kx, kept in [(3, 5, True), (N - 4, 9, True), (0, 0, True), (20, 3, False), (5, 40, False)]:
        th = 2 * np.pi * (ky * y + kx * x) / N
        v = np.cos(th)[None, None]
        S, _, _ = fno.spectral_conv(v, R)
        if not kept:
            assert np.max(np.abs(S)) < 1e-12
            continue
        # cos = (e^{i th} + e^{-i th})/2.  For kx > 0 only e^{i th} lies in the
        # half spectrum (the irfft2 doubles it): S = Re(r e^{i th}).  For kx = 0
        # both (ky, 0) and (-ky, 0) are kept and scale by r: S = Re(r) cos th.
        ref = np.real(r * np.exp(1j * th)) if kx > 0 else np.real(r) * np.cos(th)
        assert np.max(np.abs(S[0, 0] - ref)) < 1e-12, (ky, kx)


def test_spectral_conv_commutes_with_circular_shifts():
    g = np.random.default_rng(2)
    v = g.standard_normal((2, 3, N, N))
    R = g.standard_normal((fno.NMODE, 4, 3)) + 1j * g.standard_normal((fno.NMODE, 4, 3))
    S, _, _ = fno.spectral_conv(v, R)
    Ss, _, _ = fno.spectral_conv(np.roll(v, (7, -11), axis=(-2, -1)), R)
    assert np.max(np.abs(Ss - np.roll(S, (7, -11), axis=(-2, -1)))) < 1e-10 * np.max(np.abs(S))


def _params(seed=0, scale_spec=20.0):
    p = inputs.fno_init(seed)
    # larger spectral weights than the initialisation so that every path matters
    p["spec_w"] = [scale_spec * w for w in p["spec_w"]]
    return p


def _perturbed(p, key, idx, layer, h):
    q = {k: ([a.copy() for a in v] if isinstance(v, list) else v.copy()) for k, v in p.items()}
    arr = q[key][layer] if layer is not None else q[key]
    arr[idx] += h
    return q


@pytest.mark.parametrize("key,layer,idx", [
    ("lift_w", None, (3, 2)), ("lift_b", None, (5,)),
    ("spec_w", 0, (17, 2, 3)), ("spec_w", 2, (400, 31, 0)), ("spec_w", 3, (33, 5, 7)),
    ("pw_w", 1, (4, 9)), ("pw_b", 3, (1,)), ("pw_w", 3, (0, 0)),
    ("proj1_w", None, (100, 3)), ("proj1_b", None, (7,)), ("proj2_w", None, (2, 50)), ("proj2_b", None, (0,)),
])
def test_backward_matches_finite_differences(key, layer, idx):
    films = inputs.relax_films(2, seed=3)
    x = inputs.fno_features(films).astype(np.float64)
    p = _params()
    g = np.random.default_rng(4)
    tgt = g.standard_normal((2, 3, N, N))
    out, cache = fno.forward(p, x)
    grad = fno.backward(p, cache, out, tgt)
    gk = grad[key][layer] if layer is not None else grad[key]
    dL_dout = 2.0 * (out - tgt) / out.size
    for part in ((1.0,) if key != "spec_w" else (1.0, 1j)):
        # central difference of the output array (the loss itself is O(1) and
        # its change O(1e-13): differencing the outputs avoids that cancellation),
        # contracted with the exact dL/dout of the quadratic loss
        h = 1e-5 * part
        op = fno.forward(_perturbed(p, key, idx, layer, h), x)[0]
        om = fno.forward(_perturbed(p, key, idx, layer, -h), x)[0]
        fd = float(np.sum(dL_dout * (op - om))) / 2e-5
        an = gk[idx].real if part == 1.0 else gk[idx].imag
        # rounding noise of the difference: ~1e-6 of the largest entry of the group
        scale = float(np.max(np.abs(gk)))
        assert an == pytest.approx(fd, rel=1e-5, abs=1e-6 * scale), (key, layer, idx, part, an, fd)


def test_bf16_rounding_definition():
    vals = np.array([1.0, -2.5, 3.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -9, 1.0 + 3 * 2 ** -9, 0.0])
    r = fno.round_bf16(vals)
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to even -> 1; 1 + 3*2^-8 -> 1 + 2^-6 (even)
    assert list(r) == [1.0, -2.5, 3.0, 1.0, 1.0 + 2 ** -6, 1.0, 1.0 + 2 ** -7, 0.0]
    g = np.random.default_rng(5).standard_normal(10000) * 1e3
    rr = fno.round_bf16(g)
    assert np.max(np.abs(rr - g) / np.abs(g)) <= 2.0 ** -8
    assert np.all(fno.round_bf16(rr) == rr)


def test_bf16_forward_stays_close_to_float64():
    films = inputs.relax_films(2, seed=6)
    x = inputs.fno_features(films).astype(np.float64)
    p = _params()
    out64, _ = fno.forward(p, x)
    out16, _ = fno.forward(p, x, bf16=True)
    rel = np.linalg.norm(out16 - out64) / np.linalg.norm(out64)
    assert 1e-5 < rel < 3e-2
