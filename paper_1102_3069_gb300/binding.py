"""Thin ctypes binding of libmm.so (include/mm.h): same names, argument marshalling only.

Every numerical step runs in the CUDA kernels of ``csrc/``; this module only
converts Python/torch arguments into the plain pointers and sizes of the C ABI.
If the shared library has not been built the first call raises - there is no
fallback of any kind.

``Solver`` is a convenience owner of one context: it allocates the device
workspace with torch (the library itself never allocates device memory) and
forwards to the mm_* calls.
"""

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmm.so")

MM_OK, MM_EINVAL, MM_ENOMEM, MM_ECUDA = 0, -1, -2, -3
MM_ENOTCONVERGED, MM_ENONFINITE, MM_ETIMEOUT, MM_ESTATE = -4, -5, -6, -7
MM_EULER, MM_HEUN, MM_RK3, MM_RK4, MM_RKDP, MM_RKCK, MM_RK12, MM_RK23 = 1, 2, 3, 4, 5, 6, 12, 23
MM_DFT_FP32, MM_DFT_SPLIT_BF16 = 0, 1
MM_FFT_2357, MM_FFT_POW2 = 0, 1

STATUS_NAMES = {0: "MM_OK", -1: "MM_EINVAL", -2: "MM_ENOMEM", -3: "MM_ECUDA", -4: "MM_ENOTCONVERGED",
                -5: "MM_ENONFINITE", -6: "MM_ETIMEOUT", -7: "MM_ESTATE"}


class MMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class mm_stats(ctypes.Structure):
    _fields_ = [("evals", ctypes.c_longlong), ("accepted", ctypes.c_longlong), ("rejected", ctypes.c_longlong),
                ("step_index", ctypes.c_longlong), ("t", ctypes.c_double), ("dt", ctypes.c_double),
                ("last_err", ctypes.c_double), ("max_torque", ctypes.c_double), ("energy", ctypes.c_double),
                ("status", ctypes.c_int), ("done", ctypes.c_int), ("dissipation", ctypes.c_double)]


class mm_checkpoint(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("dt", ctypes.c_double), ("step_index", ctypes.c_longlong),
                ("accepted", ctypes.c_longlong), ("rejected", ctypes.c_longlong), ("evals", ctypes.c_longlong),
                ("after_reject", ctypes.c_int), ("reserved_", ctypes.c_int), ("t_internal", ctypes.c_double),
                ("dt_internal", ctypes.c_double)]


_lib = None
_vp, _dp, _i, _l, _d, _sz, _u64 = (ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_long,
                                   ctypes.c_double, ctypes.c_size_t, ctypes.c_uint64)

_SIGS = {
    "mm_init_geometry": (_i, [ctypes.POINTER(_vp), _i, _i, _i, _d, _d, _d, _i, _i, _i, _i, _vp]),
    "mm_workspace_bytes": (_sz, [_vp]),
    "mm_set_workspace": (_i, [_vp, _vp, _sz]),
    "mm_set_material": (_i, [_vp, _d, _d, _d, _dp, _d, _d, _d, _u64, _dp]),
    "mm_set_demag": (_i, [_vp, _i]),
    "mm_set_anisotropy_axes": (_i, [_vp, _vp]),
    "mm_set_max_dm": (_i, [_vp, _d]),
    "mm_set_pass_layout": (_i, [_vp, _i]),
    "mm_set_dft_precision": (_i, [_vp, _i]),
    "mm_set_fft_lengths": (_i, [_vp, _i]),
    "mm_set_cubic_anisotropy": (_i, [_vp, _d, _d, _dp, _dp]),
    "mm_set_stt": (_i, [_vp, _d, _d, _dp]),
    "mm_demag_kernel": (_i, [_vp, _dp]),
    "mm_demag_tensor_len": (_sz, [_vp]),
    "mm_eval_heff": (_i, [_vp, _vp, _vp, _vp, _dp]),
    "mm_set_thermal_clock": (_i, [_vp, _u64, _d]),
    "mm_load": (_i, [_vp, _vp, _d, _u64]),
    "mm_store": (_i, [_vp, _vp]),
    "mm_advance": (_i, [_vp, _i, _l, _d, _d, _d, _d]),
    "mm_get_stats": (_i, [_vp, ctypes.POINTER(mm_stats)]),
    "mm_step": (_i, [_vp, _vp, _i, _dp, _dp, _d, ctypes.POINTER(_i)]),
    "mm_get_state": (_i, [_vp, _vp, ctypes.POINTER(mm_checkpoint)]),
    "mm_set_state": (_i, [_vp, _vp, ctypes.POINTER(mm_checkpoint)]),
    "mm_relax": (_i, [_vp, _vp, _d, _d, _l, ctypes.POINTER(_l), _dp]),
    "mm_run_host": (_i, [_vp, _vp, _i, _l, _d, _d]),
    "mm_eval_heff_static": (_i, [_vp, _vp, _vp, _vp]),
    "mm_profile": (_i, [_vp, _i]),
    "mm_pass_times": (_i, [_vp, _dp, ctypes.POINTER(ctypes.c_longlong)]),
    "mm_last_error": (ctypes.c_char_p, [_vp]),
    "mm_destroy": (None, [_vp]),
    "mm_batch_create": (_i, [ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i, _vp]),
    "mm_batch_workspace_bytes": (_sz, [_vp]),
    "mm_batch_set_workspace": (_i, [_vp, _vp, _sz]),
    "mm_batch_load": (_i, [_vp, ctypes.POINTER(_vp)]),
    "mm_batch_store": (_i, [_vp, ctypes.POINTER(_vp)]),
    "mm_batch_advance": (_i, [_vp, _i, _l, _d, _d]),
    "mm_batch_get_stats": (_i, [_vp, ctypes.POINTER(mm_stats)]),
    "mm_batch_relax": (_i, [_vp, ctypes.POINTER(_vp), _d, _d, _l, ctypes.POINTER(_l), _dp,
                            ctypes.POINTER(_i)]),
    "mm_batch_set_tuning": (_i, [_vp, _i]),
    "mm_batch_tuning": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "mm_batch_last_error": (ctypes.c_char_p, [_vp]),
    "mm_batch_destroy": (None, [_vp]),
    "mm_fno_create": (_i, [ctypes.POINTER(_vp), _i, _vp]),
    "mm_fno_workspace_bytes": (_sz, [_vp]),
    "mm_fno_set_workspace": (_i, [_vp, _vp, _sz]),
    "mm_fno_param_count": (_sz, []),
    "mm_fno_set_params": (_i, [_vp, _vp]),
    "mm_fno_get_params": (_i, [_vp, _vp]),
    "mm_fno_train_step": (_i, [_vp, _vp, _vp, _i, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                               _dp, _vp]),
    "mm_fno_predict": (_i, [_vp, _vp, _i, _vp, _vp]),
    "mm_fno_status": (_i, [_vp]),
    "mm_fno_last_error": (ctypes.c_char_p, [_vp]),
    "mm_fno_destroy": (None, [_vp]),
    "mm_gemm_bf16": (_i, [_vp, ctypes.c_longlong, ctypes.c_longlong, _vp, ctypes.c_longlong, ctypes.c_longlong, _vp,
                          ctypes.c_longlong, ctypes.c_longlong, _i, _i, _i, _i, ctypes.c_float, _i, _vp]),
    "mm_gemm_status": (_i, [_vp]),
}


def lib():
    """Load libmm.so (built in-tree by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                               "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _ptr(x):
    """Device/host pointer of a torch tensor, a numpy array or an int address."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _check(ctx, rc):
    if rc != MM_OK:
        msg = lib().mm_last_error(ctx)
        raise MMError(rc, msg.decode() if msg else "")
    return rc


def _d3(v):
    if v is None:
        return None
    a = (ctypes.c_double * 3)(*[float(x) for x in v])
    return ctypes.cast(a, _dp), a


# ---- one-to-one wrappers (same names as the C ABI) --------------------------

def mm_init_geometry(nx, ny, nz, dx, dy, dz, pbc=(0, 0, 0), pbc_images=10, stream=None):
    ctx = _vp()
    rc = lib().mm_init_geometry(ctypes.byref(ctx), int(nx), int(ny), int(nz), float(dx), float(dy), float(dz),
                                int(bool(pbc[0])), int(bool(pbc[1])), int(bool(pbc[2])), int(pbc_images),
                                _vp(stream) if stream else None)
    if rc != MM_OK:
        raise MMError(rc, "mm_init_geometry rejected the geometry")
    return ctx


def mm_workspace_bytes(ctx):
    return int(lib().mm_workspace_bytes(ctx))


def mm_set_workspace(ctx, dev_ptr, nbytes):
    return _check(ctx, lib().mm_set_workspace(ctx, _ptr(dev_ptr), int(nbytes)))


def mm_set_material(ctx, Ms, Aex, Ku=0.0, easy_axis=(1.0, 0.0, 0.0), alpha=0.02, gamma0=0.0, temperature=0.0,
                    seed=0, B=(0.0, 0.0, 0.0)):
    u, _keep_u = _d3(easy_axis) if easy_axis is not None else (None, None)
    b, _keep_b = _d3(B)
    return _check(ctx, lib().mm_set_material(ctx, float(Ms), float(Aex), float(Ku), u, float(alpha), float(gamma0),
                                             float(temperature), int(seed) & 0xFFFFFFFFFFFFFFFF, b))


def mm_set_cubic_anisotropy(ctx, K1, K2, c1=(1.0, 0.0, 0.0), c2=(0.0, 1.0, 0.0)):
    a, _ka = _d3(c1)
    b, _kb = _d3(c2)
    return _check(ctx, lib().mm_set_cubic_anisotropy(ctx, float(K1), float(K2), a, b))


def mm_set_stt(ctx, P, xi, j=(0.0, 0.0, 0.0)):
    jj, _kj = _d3(j)
    return _check(ctx, lib().mm_set_stt(ctx, float(P), float(xi), jj))


def mm_set_anisotropy_axes(ctx, u):
    """u: device float32 tensor (3, nz, ny, nx) of unit easy axes, or None."""
    return _check(ctx, lib().mm_set_anisotropy_axes(ctx, _ptr(u)))


MM_LAYOUT_AUTO, MM_LAYOUT_FUSED, MM_LAYOUT_SPLIT, MM_LAYOUT_CLUSTER = 0, 1, 2, 3


def mm_set_pass_layout(ctx, layout):
    return _check(ctx, lib().mm_set_pass_layout(ctx, int(layout)))


def mm_set_dft_precision(ctx, mode):
    return _check(ctx, lib().mm_set_dft_precision(ctx, int(mode)))


def mm_set_fft_lengths(ctx, mode):
    return _check(ctx, lib().mm_set_fft_lengths(ctx, int(mode)))


def mm_set_max_dm(ctx, max_dm):
    return _check(ctx, lib().mm_set_max_dm(ctx, float(max_dm)))


def mm_set_demag(ctx, enabled):
    return _check(ctx, lib().mm_set_demag(ctx, int(bool(enabled))))


def mm_demag_tensor_len(ctx):
    return int(lib().mm_demag_tensor_len(ctx))


def mm_demag_kernel(ctx, dump=False):
    """Build the kernel; with dump=True return the FP64 real-space octant as numpy."""
    if dump:
        out = np.zeros(mm_demag_tensor_len(ctx), dtype=np.float64)
        _check(ctx, lib().mm_demag_kernel(ctx, out.ctypes.data_as(_dp)))
        return out
    _check(ctx, lib().mm_demag_kernel(ctx, None))
    return None


def mm_eval_heff(ctx, m, h_out=None, torque_out=None, energy=False):
    e = ctypes.c_double(0.0)
    _check(ctx, lib().mm_eval_heff(ctx, _ptr(m), _ptr(h_out), _ptr(torque_out), ctypes.byref(e) if energy else None))
    return e.value if energy else None


def mm_eval_heff_static(ctx, m, h_out=None, torque_out=None):
    """Allocation-free evaluation: scratch in the library's static device array."""
    return _check(ctx, lib().mm_eval_heff_static(ctx, _ptr(m), _ptr(h_out), _ptr(torque_out)))


def mm_set_thermal_clock(ctx, step_index, dt_s):
    return _check(ctx, lib().mm_set_thermal_clock(ctx, int(step_index), float(dt_s)))


def mm_load(ctx, m, t0_s=0.0, step_index=0):
    return _check(ctx, lib().mm_load(ctx, _ptr(m), float(t0_s), int(step_index)))


def mm_store(ctx, m):
    return _check(ctx, lib().mm_store(ctx, _ptr(m)))


def mm_advance(ctx, method, nsteps, dt_s=0.0, tol=1e-6, t_end_s=0.0, torque_tol=0.0):
    return _check(ctx, lib().mm_advance(ctx, int(method), int(nsteps), float(dt_s), float(tol), float(t_end_s),
                                        float(torque_tol)))


def mm_get_stats(ctx):
    s = mm_stats()
    _check(ctx, lib().mm_get_stats(ctx, ctypes.byref(s)))
    return {f: getattr(s, f) for f, _ in mm_stats._fields_}


def mm_get_state(ctx, m=None):
    """Checkpoint: copies the state into m (device tensor, optional); returns the scalars as a dict."""
    c = mm_checkpoint()
    _check(ctx, lib().mm_get_state(ctx, _ptr(m), ctypes.byref(c)))
    return {f: getattr(c, f) for f, _ in mm_checkpoint._fields_ if f != "reserved_"}


def mm_set_state(ctx, m, cp):
    c = mm_checkpoint(**{k: cp[k] for k in ("t", "dt", "step_index", "accepted", "rejected", "evals",
                                            "after_reject", "t_internal", "dt_internal") if k in cp})
    return _check(ctx, lib().mm_set_state(ctx, _ptr(m), ctypes.byref(c)))


def mm_step(ctx, m, method, t_s, dt_s, tol=1e-6):
    t = ctypes.c_double(t_s)
    dt = ctypes.c_double(dt_s)
    acc = ctypes.c_int(0)
    _check(ctx, lib().mm_step(ctx, _ptr(m), int(method), ctypes.byref(t), ctypes.byref(dt), float(tol),
                              ctypes.byref(acc)))
    return bool(acc.value), t.value, dt.value


def mm_relax(ctx, m, torque_tol=1e-4, err_tol=1e-5, max_steps=100000):
    steps = ctypes.c_long(0)
    tq = ctypes.c_double(0.0)
    rc = lib().mm_relax(ctx, _ptr(m), float(torque_tol), float(err_tol), int(max_steps), ctypes.byref(steps),
                        ctypes.byref(tq))
    _check(ctx, rc)
    return steps.value, tq.value


def mm_run_host(ctx, m_host, method, nsteps, dt_s=0.0, tol=1e-6):
    return _check(ctx, lib().mm_run_host(ctx, _ptr(m_host), int(method), int(nsteps), float(dt_s), float(tol)))


PASS_NAMES = ["k_xfwd", "k_colconv_y", "k_yfwd", "k_colconv_z", "k_yinv", "k_xinv_local", "k_combine2", "k_local",
              "k_xinv_local_fused", "k_xinv_h", "k_local_h", "k_xfwd_next", "k_small", "k_yzconv"]
NPASS = len(PASS_NAMES)


def mm_profile(ctx, enable):
    return _check(ctx, lib().mm_profile(ctx, int(bool(enable))))


def mm_pass_times(ctx):
    ms = (ctypes.c_double * NPASS)()
    n = (ctypes.c_longlong * NPASS)()
    _check(ctx, lib().mm_pass_times(ctx, ms, n))
    return {PASS_NAMES[i]: {"ms_total": ms[i], "launches": n[i],
                            "ms_per_launch": ms[i] / n[i] if n[i] else 0.0} for i in range(NPASS) if n[i]}


def pass_times(ctx, fn):
    """Run fn() with per-pass event timing on and return mm_pass_times."""
    mm_profile(ctx, True)
    try:
        fn()
        return mm_pass_times(ctx)
    finally:
        mm_profile(ctx, False)


def mm_last_error(ctx):
    msg = lib().mm_last_error(ctx)
    return msg.decode() if msg else ""


def mm_destroy(ctx):
    lib().mm_destroy(ctx)


# ---- batched ensembles -------------------------------------------------------

def _bcheck(b, rc):
    if rc != MM_OK:
        msg = lib().mm_batch_last_error(b)
        raise MMError(rc, msg.decode() if msg else "")
    return rc


def _ptr_array(xs):
    return (_vp * len(xs))(*[_ptr(x) for x in xs])


def mm_batch_create(ctxs, stream=None):
    b = _vp()
    arr = (_vp * len(ctxs))(*[c.value if isinstance(c, _vp) else c for c in ctxs])
    rc = lib().mm_batch_create(ctypes.byref(b), arr, len(ctxs), _vp(stream) if stream else None)
    if rc != MM_OK:
        raise MMError(rc, "mm_batch_create rejected a context")
    return b


def mm_batch_workspace_bytes(b):
    return int(lib().mm_batch_workspace_bytes(b))


def mm_batch_set_workspace(b, dev_ptr, nbytes):
    return _bcheck(b, lib().mm_batch_set_workspace(b, _ptr(dev_ptr), int(nbytes)))


def mm_batch_load(b, ms):
    return _bcheck(b, lib().mm_batch_load(b, _ptr_array(ms)))


def mm_batch_store(b, ms):
    return _bcheck(b, lib().mm_batch_store(b, _ptr_array(ms)))


def mm_batch_advance(b, method, nsteps, dt_s=0.0, tol=1e-6):
    return _bcheck(b, lib().mm_batch_advance(b, int(method), int(nsteps), float(dt_s), float(tol)))


def mm_batch_get_stats(b, n):
    arr = (mm_stats * n)()
    _bcheck(b, lib().mm_batch_get_stats(b, arr))
    return [{f: getattr(s, f) for f, _ in mm_stats._fields_} for s in arr]


def mm_batch_relax(b, ms, torque_tol=1e-4, err_tol=1e-5, max_steps=100000, check=True):
    """Returns (rc, steps per sample, torque per sample, number converged)."""
    n = len(ms)
    steps = (_l * n)()
    tq = (ctypes.c_double * n)()
    conv = _i(0)
    rc = lib().mm_batch_relax(b, _ptr_array(ms), float(torque_tol), float(err_tol), int(max_steps), steps,
                              ctypes.cast(tq, _dp), ctypes.byref(conv))
    if check and rc not in (MM_OK, MM_ENOTCONVERGED):
        _bcheck(b, rc)
    return rc, list(steps), list(tq), conv.value


def mm_batch_set_tuning(b, mode):
    return _bcheck(b, lib().mm_batch_set_tuning(b, int(mode)))


def mm_batch_tuning(b):
    """(launch groups, groups with two register budgets, groups running the second)."""
    g, t, a = _i(0), _i(0), _i(0)
    _bcheck(b, lib().mm_batch_tuning(b, ctypes.byref(g), ctypes.byref(t), ctypes.byref(a)))
    return g.value, t.value, a.value


def mm_batch_last_error(b):
    msg = lib().mm_batch_last_error(b)
    return msg.decode() if msg else ""


def mm_batch_destroy(b):
    lib().mm_batch_destroy(b)


class Batch:
    """An ensemble of Solvers stepped together (all on one stream)."""

    def __init__(self, solvers, stream):
        import torch
        self.solvers = list(solvers)
        self.b = mm_batch_create([s.ctx for s in self.solvers], stream)
        nbytes = mm_batch_workspace_bytes(self.b)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = self.workspace.data_ptr()
        mm_batch_set_workspace(self.b, (base + 255) // 256 * 256, nbytes)

    def __del__(self):
        try:
            if getattr(self, "b", None) is not None:
                mm_batch_destroy(self.b)
                self.b = None
        except Exception:
            pass


# ---- convenience owner ------------------------------------------------------

class Solver:
    """One geometry + material on the current CUDA device; workspace from torch.

    shape = (nx, ny, nz), cell = (dx, dy, dz) in m; material keywords as in
    mm_set_material.  ``demag=False`` disables the magnetostatic term.
    """

    def __init__(self, shape, cell, pbc=(0, 0, 0), images=10, demag=True, stream=None, tensor=True,
                 dft_precision=None, fft_lengths=None, **material):
        import torch
        self.torch = torch
        self.shape = tuple(int(v) for v in shape)
        self.cell = tuple(float(v) for v in cell)
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        self.ctx = mm_init_geometry(*self.shape, *self.cell, pbc, images, stream)
        if fft_lengths is not None:
            mm_set_fft_lengths(self.ctx, fft_lengths)
        if dft_precision is not None:
            mm_set_dft_precision(self.ctx, dft_precision)
        nbytes = mm_workspace_bytes(self.ctx)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = self.workspace.data_ptr()
        aligned = (base + 255) // 256 * 256
        mm_set_workspace(self.ctx, aligned, nbytes)
        mm_set_material(self.ctx, **material)
        mm_set_demag(self.ctx, demag)
        self.tensor = None
        if demag:
            self.tensor = mm_demag_kernel(self.ctx, dump=tensor)

    @property
    def mshape(self):
        nx, ny, nz = self.shape
        return (3, nz, ny, nx)

    def set_material(self, **material):
        mm_set_material(self.ctx, **material)

    def heff(self, m, torque=False, energy=False):
        h = self.torch.empty_like(m)
        tq = self.torch.empty_like(m) if torque else None
        e = mm_eval_heff(self.ctx, m, h, tq, energy)
        return h, tq, e

    def close(self):
        if self.ctx is not None:
            mm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- learned warm start (include/mm_fno.h) ----------------------------------

def _fcheck(f, rc):
    if rc != MM_OK:
        msg = lib().mm_fno_last_error(f)
        raise MMError(rc, msg.decode() if msg else "")
    return rc


def mm_fno_create(max_batch, stream=None):
    f = _vp()
    rc = lib().mm_fno_create(ctypes.byref(f), int(max_batch), stream)
    if rc != MM_OK:
        raise MMError(rc, "mm_fno_create")
    return f


def mm_fno_workspace_bytes(f):
    return int(lib().mm_fno_workspace_bytes(f))


def mm_fno_set_workspace(f, ptr, nbytes):
    return _fcheck(f, lib().mm_fno_set_workspace(f, _ptr(ptr), int(nbytes)))


def mm_fno_param_count():
    return int(lib().mm_fno_param_count())


def mm_fno_set_params(f, params):
    return _fcheck(f, lib().mm_fno_set_params(f, _ptr(params)))


def mm_fno_get_params(f, params):
    return _fcheck(f, lib().mm_fno_get_params(f, _ptr(params)))


def mm_fno_train_step(f, x, target, batch, lr, beta1=0.9, beta2=0.999, eps=1e-8, want_loss=True, grad_out=None):
    loss = ctypes.c_double(0.0)
    _fcheck(f, lib().mm_fno_train_step(f, _ptr(x), _ptr(target), int(batch), float(lr), float(beta1), float(beta2),
                                       float(eps), ctypes.byref(loss) if want_loss else None, _ptr(grad_out)))
    return loss.value if want_loss else None


def mm_fno_predict(f, x, batch, m_out=None, raw_out=None):
    return _fcheck(f, lib().mm_fno_predict(f, _ptr(x), int(batch), _ptr(m_out), _ptr(raw_out)))


def mm_fno_status(f):
    return lib().mm_fno_status(f)


def mm_fno_last_error(f):
    msg = lib().mm_fno_last_error(f)
    return msg.decode() if msg else ""


def mm_fno_destroy(f):
    lib().mm_fno_destroy(f)


def mm_gemm_bf16(a, lda, a_batch, b, ldb, b_batch, c, ldc, c_batch, m, n, k, batch=1, alpha=1.0, beta=0, stream=None):
    rc = lib().mm_gemm_bf16(_ptr(a), int(lda), int(a_batch), _ptr(b), int(ldb), int(b_batch), _ptr(c), int(ldc),
                            int(c_batch), int(m), int(n), int(k), int(batch), float(alpha), int(beta), stream)
    if rc != MM_OK:
        raise MMError(rc, "mm_gemm_bf16: bad sizes, strides or alignment")
    return rc


def mm_gemm_status(stream=None):
    return lib().mm_gemm_status(stream)


# Flat parameter vector of include/mm_fno.h <-> the dict form of the seeded
# initialisation (inputs.fno_init): marshalling only.
FNO_SHAPES = [("lift_w", (32, 16)), ("lift_b", (32,)), ("spec_w", (4, 2, 512, 32, 32)), ("pw_w", (4, 32, 32)),
              ("pw_b", (4, 32)), ("proj1_w", (128, 32)), ("proj1_b", (128,)), ("proj2_w", (3, 128)),
              ("proj2_b", (3,))]


def fno_pack(p):
    """dict (numpy float64, spec_w a list of 4 complex [512][32][32]) -> flat float32 numpy array."""
    parts = []
    for name, shape in FNO_SHAPES:
        v = p[name]
        if name == "spec_w":
            v = np.stack([np.stack([np.real(w), np.imag(w)]) for w in v])
        elif isinstance(v, list):
            v = np.stack(v)
        parts.append(np.asarray(v, dtype=np.float32).reshape(-1))
    return np.concatenate(parts)


def fno_unpack(flat):
    flat = np.asarray(flat, dtype=np.float64)
    out, off = {}, 0
    for name, shape in FNO_SHAPES:
        n = int(np.prod(shape))
        v = flat[off:off + n].reshape(shape)
        off += n
        if name == "spec_w":
            v = [v[l, 0] + 1j * v[l, 1] for l in range(4)]
        elif name in ("pw_w", "pw_b"):
            v = [v[l] for l in range(4)]
        out[name] = v
    return out


class Fno:
    """The warm-start operator on the current CUDA device; workspace from torch."""

    def __init__(self, max_batch, stream=None):
        import torch
        self.torch = torch
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        self.f = mm_fno_create(max_batch, stream)
        nbytes = mm_fno_workspace_bytes(self.f)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = self.workspace.data_ptr()
        mm_fno_set_workspace(self.f, (base + 255) // 256 * 256, nbytes)
        self.nparam = mm_fno_param_count()

    def set_params(self, p):
        flat = p if isinstance(p, np.ndarray) else fno_pack(p)
        t = self.torch.from_numpy(np.ascontiguousarray(flat, dtype=np.float32)).cuda()
        mm_fno_set_params(self.f, t)
        self.torch.cuda.synchronize()

    def get_params(self):
        t = self.torch.empty(self.nparam, dtype=self.torch.float32, device="cuda")
        mm_fno_get_params(self.f, t)
        return t.cpu().numpy()

    def close(self):
        if getattr(self, "f", None) is not None:
            mm_fno_destroy(self.f)
            self.f = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
