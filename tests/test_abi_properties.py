"""Property tests of the geometry rules of include/mm.h through the real C
ABI, on the host (no device call): mm_init_geometry accepts exactly the
documented shapes, and the sizes it reports follow the documented layout."""

import pytest

from paper_1102_3069_gb300 import binding as B

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st   # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    import os
    if not os.path.exists(B.LIB_PATH):
        from paper_1102_3069_gb300 import build
        build.build()


# lengths r * 2^l with an odd factor r that have compiled passes (every axis)
ODD = {r << l for r, ls in ((3, range(6, 11)), (5, range(6, 10)), (7, range(6, 10))) for l in ls}


def _accepted(n, periodic, axis):
    if n < 1:
        return False
    if periodic:
        return (n <= 4096 and (n & (n - 1)) == 0) or n in ODD
    return n <= 2048


def _try(nx, ny, nz, pbc):
    try:
        return B.mm_init_geometry(nx, ny, nz, 4e-9, 3e-9, 2e-9, pbc=pbc, pbc_images=2)
    except B.MMError as e:
        assert e.code == B.MM_EINVAL
        return None


sizes = st.one_of(st.integers(-3, 70), st.integers(2030, 2060), st.integers(4090, 4100),
                  st.sampled_from([1, 2, 64, 512, 1024, 2048, 4096, 8192, 48, 96, 192, 320, 448, 1280, 3072, 3584,
                                   6144]))


@settings(max_examples=400, deadline=None)
@given(nx=sizes, ny=sizes, nz=sizes, pbc=st.tuples(st.booleans(), st.booleans(), st.booleans()))
def test_geometry_accepted_exactly_as_documented(nx, ny, nz, pbc):
    ctx = _try(nx, ny, nz, tuple(int(p) for p in pbc))
    expect = all(_accepted(n, p, a) for a, (n, p) in enumerate(zip((nx, ny, nz), pbc)))
    assert (ctx is not None) == expect, (nx, ny, nz, pbc)
    if ctx is None:
        return
    try:
        # tensor dump: six components, O = n on an open axis, n/2 + 1 on a periodic one
        o = [n // 2 + 1 if p else n for n, p in zip((nx, ny, nz), pbc)]
        assert B.mm_demag_tensor_len(ctx) == 6 * o[0] * o[1] * o[2]
        # the workspace holds at least the twelve stage arrays of 3 floats per cell
        assert B.mm_workspace_bytes(ctx) >= 12 * 12 * nx * ny * nz
        assert B.mm_workspace_bytes(ctx) % 256 == 0
    finally:
        B.mm_destroy(ctx)


@settings(max_examples=60, deadline=None)
@given(n=st.integers(1, 2047))
def test_workspace_never_shrinks_as_an_open_axis_grows(n):
    """Up to the twiddle table of an odd factor (at most 7 x 4096 complex
    values), which only lengths with that factor carry."""
    a = B.mm_init_geometry(n, 8, 1, 4e-9, 4e-9, 4e-9)
    b = B.mm_init_geometry(n + 1, 8, 1, 4e-9, 4e-9, 4e-9)
    try:
        assert B.mm_workspace_bytes(a) <= B.mm_workspace_bytes(b) + 7 * 4096 * 8
    finally:
        B.mm_destroy(a)
        B.mm_destroy(b)


@settings(max_examples=100, deadline=None)
@given(d=st.tuples(*[st.one_of(st.floats(-1e-8, 1e-8), st.just(float("nan")), st.just(float("inf")))] * 3))
def test_cell_sizes_must_be_positive_and_finite(d):
    ok = all(v > 0 and v != float("inf") for v in d)
    try:
        ctx = B.mm_init_geometry(8, 8, 1, *d)
    except B.MMError as e:
        assert not ok and e.code == B.MM_EINVAL
        return
    assert ok
    B.mm_destroy(ctx)
