"""Fourier neural operator (FNO) of the learned relaxation warm start.

TEST INFRASTRUCTURE ONLY: plain numpy, read by the tests, __graft_entry__.smoke()
and bench.py's CPU legs; the CUDA path never imports it.

The paper relaxes every standard problem from a start state with the plain
solver (Sec. 4; the scripted relax() of Sec. 6).  The warm start replaces the
random start by the prediction of a Fourier neural operator (Li et al.,
"Fourier neural operator for parametric partial differential equations",
ICLR 2021) trained on relaxed states the solver produced; the solver then
finishes the relaxation.  The operator, written out here step by step:

  grid       128 x 128 cells, p = y*128 + x
  input      per cell 16 channels (the seeded input generator's fno_features:
             material, field and cell position; 8 used, the rest zero)
  lift       v0 = Wl in + bl                                   (16 -> 32)
  layer l    z_l = S_l(v_l) + Wp_l v_l + bp_l,  v_{l+1} = gelu(z_l)  (l = 0..3;
             the last layer has no gelu: v4 = z_3)
  spectral   S(v) = irfft2 of [R_m Vhat_m on the kept modes, 0 elsewhere],
             Vhat = rfft2(v), kept modes kx in 0..15, ky in 0..15 and 112..127
             (16 per axis and sign: 512 modes), R_m a complex 32 x 32 matrix
  project    h = gelu(Q1 v4 + q1)  (32 -> 128),  out = Q2 h + q2  (128 -> 3)
  loss       mean over cells, components and samples of (out - m_relaxed)^2
  gelu(z)    z/2 (1 + erf(z/sqrt 2))

Precision (bf16=True): every operand of a product - weights, the input
features, activations, the kept spectra before and after the mode mixing,
and the gradients fed back through a product - is rounded to bfloat16
(round to nearest even); sums and everything else stay in higher precision.
This is the precision of the GPU kernels (BF16 operands, FP32 accumulation).
bf16=False computes everything in float64.

Array layouts: activations (B, C, 128, 128); spectral weights R (512, 32, 32)
complex indexed [mode, out, in] with mode = ix*32 + jy (ix = kx, jy indexes ky
as 0..15, 112..127).

Pins (tests/test_oracle_fno.py): the backward pass equals central finite
differences of the forward pass; the spectral convolution with R = identity
equals the low-pass projection written as an explicit sum of the kept
Fourier modes; the spectral convolution commutes with circular shifts; the
bf16 rounding matches the bit-level definition.
"""

import math

import numpy as np
from scipy.special import erf

N = 128
NP = N * N
WIDTH = 32
MODES = 16
CIN = 16
CHID = 128
COUT = 3
NMODE = MODES * 2 * MODES      # 512
KX = np.arange(MODES)
KY = np.concatenate([np.arange(MODES), np.arange(N - MODES, N)])


def mode_ky_kx():
    """(ky, kx) of every mode, mode = ix*32 + jy."""
    ky = np.tile(KY, MODES)
    kx = np.repeat(KX, 2 * MODES)
    return ky, kx


def round_bf16(a):
    """Round float values to the nearest bfloat16 (ties to even), returned as float64."""
    a = np.asarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _rb(a, on):
    if np.iscomplexobj(a):
        if not on:
            return np.asarray(a, dtype=np.complex128)
        return round_bf16(a.real) + 1j * round_bf16(a.imag)
    return round_bf16(a) if on else np.asarray(a, dtype=np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def _kept(Vh):
    """(B, C, N, N/2+1) half spectrum -> (B, C, 512) kept modes."""
    sub = Vh[:, :, KY, :][:, :, :, KX]                   # (B, C, 32 ky, 16 kx)
    return np.transpose(sub, (0, 1, 3, 2)).reshape(Vh.shape[0], Vh.shape[1], NMODE)


def _place(Um):
    """(B, C, 512) -> (B, C, N, N/2+1) half spectrum, zero outside the kept modes."""
    B, C = Um.shape[:2]
    Uh = np.zeros((B, C, N, N // 2 + 1), dtype=np.complex128)
    blk = np.transpose(Um.reshape(B, C, MODES, 2 * MODES), (0, 1, 3, 2))    # (B, C, 32 ky, 16 kx)
    Uh[:, :, KY[:, None], KX[None, :]] = blk
    return Uh


def spectral_conv(v, R, bf16=False):
    """S(v) and the intermediates (kept input spectrum, mixed spectrum)."""
    Vm = _rb(_kept(np.fft.rfft2(v)), bf16)
    Um = _rb(np.einsum("moi,bim->bom", _rb(R, bf16), Vm), bf16)
    return np.fft.irfft2(_place(Um), s=(N, N)), Vm, Um


def forward(params, x, bf16=False):
    """x: (B, 16, N, N) input features.  Returns (out (B, 3, N, N), cache)."""
    P = params
    c = {"x": _rb(x, bf16)}
    v = _rb(np.einsum("oi,bihw->bohw", _rb(P["lift_w"], bf16), c["x"]) + P["lift_b"][None, :, None, None], bf16)
    c["v"] = [v]
    c["z"], c["Vm"] = [], []
    for l in range(4):
        S, Vm, _ = spectral_conv(v, P["spec_w"][l], bf16)
        z = S + np.einsum("oi,bihw->bohw", _rb(P["pw_w"][l], bf16), v) + P["pw_b"][l][None, :, None, None]
        c["z"].append(z)
        c["Vm"].append(Vm)
        v = _rb(gelu(z) if l < 3 else z, bf16)
        c["v"].append(v)
    hp = np.einsum("oi,bihw->bohw", _rb(P["proj1_w"], bf16), v) + P["proj1_b"][None, :, None, None]
    h = _rb(gelu(hp), bf16)
    out = np.einsum("oi,bihw->bohw", _rb(P["proj2_w"], bf16), h) + P["proj2_b"][None, :, None, None]
    c["hp"], c["h"] = hp, h
    return out, c


def loss(out, target):
    return float(np.mean((out - target) ** 2))


def backward(params, cache, out, target, bf16=False):
    """Gradients of loss(out, target) for every parameter (same keys and shapes)."""
    P = params
    g = {}
    nel = out.size
    dout = _rb(2.0 * (out - target) / nel, bf16)
    h = cache["h"]
    g["proj2_w"] = np.einsum("bohw,bihw->oi", dout, h)
    g["proj2_b"] = dout.sum(axis=(0, 2, 3))
    dh = np.einsum("oi,bohw->bihw", _rb(P["proj2_w"], bf16), dout)
    dhp = _rb(dh * gelu_grad(cache["hp"]), bf16)
    v4 = cache["v"][4]
    g["proj1_w"] = np.einsum("bohw,bihw->oi", dhp, v4)
    g["proj1_b"] = dhp.sum(axis=(0, 2, 3))
    dv = np.einsum("oi,bohw->bihw", _rb(P["proj1_w"], bf16), dhp)
    ky, kx = mode_ky_kx()
    wk = np.where(kx == 0, 1.0, 2.0)                      # Hermitian weight of irfft2
    g["spec_w"], g["pw_w"], g["pw_b"] = [None] * 4, [None] * 4, [None] * 4
    for l in range(3, -1, -1):
        z = cache["z"][l]
        dz = _rb(dv if l == 3 else dv * gelu_grad(z), bf16)
        vl = cache["v"][l]
        g["pw_w"][l] = np.einsum("bohw,bihw->oi", dz, vl)
        g["pw_b"][l] = dz.sum(axis=(0, 2, 3))
        dv = np.einsum("oi,bohw->bihw", _rb(P["pw_w"][l], bf16), dz)
        # S(v) = irfft2(place(Um)): d/dUm (re + i im) = (w(kx)/N^2) rfft2(dz) on the kept modes
        dUm = _rb(_kept(np.fft.rfft2(dz)) * (wk / NP)[None, None, :], bf16)
        Vm = cache["Vm"][l]
        R = _rb(P["spec_w"][l], bf16)
        g["spec_w"][l] = np.einsum("bom,bim->moi", dUm, np.conj(Vm))
        dVm = _rb(np.einsum("moi,bom->bim", np.conj(R), dUm), bf16)
        # Vm = rfft2(v) on the kept modes: dv[p] = sum_m Re(dVm e^{+i theta_m p})
        dv = dv + np.fft.irfft2(_place(dVm / wk[None, None, :]), s=(N, N)) * NP
    dv = _rb(dv, bf16)
    g["lift_w"] = np.einsum("bohw,bihw->oi", dv, cache["x"])
    g["lift_b"] = dv.sum(axis=(0, 2, 3))
    return g
