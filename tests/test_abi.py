"""The C ABI library loads and exports every entry point that include/mm.h
declares; host-side argument checks work without a GPU (no compute calls)."""

import ctypes
import os
import re

import pytest

from paper_1102_3069_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _ensure_built():
    if not os.path.exists(B.LIB_PATH):
        from paper_1102_3069_gb300 import build
        build.build()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(mm_\w+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported():
    _ensure_built()
    lib = ctypes.CDLL(B.LIB_PATH)
    declared = _declared()
    assert len(declared) >= 18
    for name in declared:
        assert hasattr(lib, name), name
    # the binding wraps every one of them under the same name
    assert declared <= set(B.exported_symbols()) | {n for n in declared if hasattr(B, n)}
    for name in declared:
        assert hasattr(B, name), name


def test_geometry_validation_on_host():
    _ensure_built()
    for bad in [(0, 4, 1), (4, -1, 1), (4097, 1, 1), (2049, 1, 1)]:
        with pytest.raises(B.MMError) as e:
            B.mm_init_geometry(*bad, 1e-9, 1e-9, 1e-9)
        assert e.value.code == B.MM_EINVAL
    with pytest.raises(B.MMError):
        B.mm_init_geometry(6, 4, 1, 1e-9, 1e-9, 1e-9, pbc=(1, 0, 0))      # periodic axis not a power of two
    with pytest.raises(B.MMError):
        B.mm_init_geometry(4, 4, 1, 0.0, 1e-9, 1e-9)


def test_workspace_size_and_material_checks_on_host():
    _ensure_built()
    ctx = B.mm_init_geometry(64, 16, 1, 4e-9, 4e-9, 4e-9)
    try:
        n = B.mm_workspace_bytes(ctx)
        # at least the 11 stage arrays of 3 floats per cell and the kernel octant
        assert n >= 11 * 3 * 4 * 64 * 16 + 4 * 65 * 17 * 4
        assert B.mm_demag_tensor_len(ctx) == 6 * 64 * 16
        with pytest.raises(B.MMError) as e:
            B.mm_set_material(ctx, Ms=-1.0, Aex=1e-11)
        assert e.value.code == B.MM_EINVAL
        with pytest.raises(B.MMError) as e:
            B.mm_set_material(ctx, Ms=8e5, Aex=1e-11, Ku=1e3, easy_axis=(0.0, 0.0, 0.0))
        assert e.value.code == B.MM_EINVAL
        B.mm_set_material(ctx, Ms=8e5, Aex=1.3e-11)
        with pytest.raises(B.MMError) as e:            # no workspace yet
            B.mm_eval_heff(ctx, 0, 0)
        assert e.value.code == B.MM_ENOMEM
        assert "workspace" in B.mm_last_error(ctx)
    finally:
        B.mm_destroy(ctx)
    B.lib().mm_destroy(None)


def test_larger_grids_need_larger_workspaces():
    _ensure_built()
    a = B.mm_init_geometry(32, 32, 1, 4e-9, 4e-9, 4e-9)
    b = B.mm_init_geometry(1024, 1024, 1, 4e-9, 4e-9, 2e-9)
    c = B.mm_init_geometry(256, 256, 64, 3e-9, 3e-9, 3e-9, pbc=(1, 1, 0))
    try:
        assert B.mm_workspace_bytes(a) < B.mm_workspace_bytes(b) < B.mm_workspace_bytes(c)
        # 1024^2 film: 11 stage arrays (12 B/cell) + spectrum + kernel, well under 1 GB
        assert B.mm_workspace_bytes(b) < 400 * 2 ** 20
    finally:
        for x in (a, b, c):
            B.mm_destroy(x)


def test_option_calls_check_their_arguments_on_host():
    """The option and checkpoint calls reject bad arguments before any device
    work (no GPU needed)."""
    _ensure_built()
    ctx = B.mm_init_geometry(64, 16, 1, 4e-9, 4e-9, 4e-9)
    try:
        for bad in (-1, 4, 7):
            with pytest.raises(B.MMError) as e:
                B.mm_set_pass_layout(ctx, bad)
            assert e.value.code == B.MM_EINVAL
        for layout in (B.MM_LAYOUT_AUTO, B.MM_LAYOUT_FUSED, B.MM_LAYOUT_SPLIT, B.MM_LAYOUT_CLUSTER):
            B.mm_set_pass_layout(ctx, layout)
        # the one-launch cluster evaluation: 2-D grids whose half spectrum fits 16 CTAs
        for shape in ((8, 8, 2), (600, 7, 1), (300, 300, 1)):
            c3 = B.mm_init_geometry(*shape, 4e-9, 4e-9, 4e-9)
            try:
                with pytest.raises(B.MMError) as e:
                    B.mm_set_pass_layout(c3, B.MM_LAYOUT_CLUSTER)
                assert e.value.code == B.MM_EINVAL
            finally:
                B.mm_destroy(c3)
        for bad in (-0.1, 1.5, float("nan")):
            with pytest.raises(B.MMError) as e:
                B.mm_set_max_dm(ctx, bad)
            assert e.value.code == B.MM_EINVAL
        B.mm_set_max_dm(ctx, 0.02)
        B.mm_set_max_dm(ctx, 0.0)
        with pytest.raises(B.MMError) as e:            # not float aligned
            B.mm_set_anisotropy_axes(ctx, 0x1002)
        assert e.value.code == B.MM_EINVAL
        B.mm_set_anisotropy_axes(ctx, None)
        with pytest.raises(B.MMError) as e:            # nothing loaded to checkpoint
            B.mm_get_state(ctx)
        assert e.value.code == B.MM_ESTATE
        with pytest.raises(B.MMError) as e:            # no workspace to restore into
            B.mm_set_state(ctx, 0x1000, dict(t=0.0, dt=1e-13, step_index=0, accepted=0, rejected=0, evals=0,
                                             after_reject=0))
        assert e.value.code == B.MM_ENOMEM
        with pytest.raises(B.MMError) as e:            # a context without workspace cannot join a batch
            B.mm_batch_create([ctx])
        assert e.value.code == B.MM_EINVAL
    finally:
        B.mm_destroy(ctx)
    b = ctypes.c_void_p()
    assert B.lib().mm_batch_create(ctypes.byref(b), None, 0, None) == B.MM_EINVAL
    assert B.mm_batch_workspace_bytes(None) == 0
    B.lib().mm_batch_destroy(None)


def test_fft_length_choice_on_the_host():
    """An open axis of 600 cells pads to 1280 = 5 * 256 by default and to 2048
    with MM_FFT_POW2 (the choice moves the workspace size); a periodic axis
    of 192 = 3 * 64 cells keeps its odd factor and refuses MM_FFT_POW2."""
    _ensure_built()
    a = B.mm_init_geometry(600, 7, 1, 4e-9, 4e-9, 4e-9)
    b = B.mm_init_geometry(600, 7, 1, 4e-9, 4e-9, 4e-9)
    c = B.mm_init_geometry(192, 8, 1, 4e-9, 4e-9, 4e-9, pbc=(1, 0, 0))
    try:
        B.mm_set_fft_lengths(b, B.MM_FFT_POW2)
        # spectrum rows: (1280/2 + 1) against (2048/2 + 1) complex values per row
        assert B.mm_workspace_bytes(b) > B.mm_workspace_bytes(a)
        B.mm_set_fft_lengths(b, B.MM_FFT_2357)
        assert B.mm_workspace_bytes(b) == B.mm_workspace_bytes(a)
        with pytest.raises(B.MMError) as e:
            B.mm_set_fft_lengths(c, B.MM_FFT_POW2)
        assert e.value.code == B.MM_EINVAL
        with pytest.raises(B.MMError):
            B.mm_set_fft_lengths(a, 7)
    finally:
        for x in (a, b, c):
            B.mm_destroy(x)
