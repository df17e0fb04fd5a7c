"""Thin ctypes binding of libfr3d.so (include/fr3d.h): argument marshalling only.

Every computation runs in the library's CUDA kernels; this module converts Python
values and torch CUDA tensors (device memory and streams only) into the C ABI's
pointers and sizes, and raises Fr3dError on a negative status.  There is no
fallback: if the library is missing, ``load()`` raises.
"""

from __future__ import annotations

import ctypes as ct
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libfr3d.so")

OK = 0
PREC_FP32, PREC_FP64, PREC_BF16TC, PREC_BF16X3 = 0, 1, 2, 3
ALPHA_FIXED, ALPHA_DISCREPANCY, ALPHA_GIVEN, ALPHA_LEARNED = 0, 1, 2, 3
MAX_BANDS = 16
OUT_ZETA, OUT_XI = 0, 1
RA_TIKHONOV, RA_TSVD = 0, 1
INFO_ALPHA_NONE_SATISFIES, INFO_ALPHA_ALL_SATISFY, INFO_NONFINITE, INFO_LEARNED_OUT_OF_RANGE = 1, 2, 4, 8
INFO_TIMEOUT = 16
MAX_HIDDEN = 96
K_DZ_INV_R, K_INV_R = 0, 1
MAX_ALPHAS = 128
MAX_SOURCE_POINTS = 256

_dp = ct.POINTER(ct.c_double)


class Geometry(ct.Structure):
    _fields_ = [("nx", ct.c_int), ("ny", ct.c_int), ("x0", ct.c_double), ("y0", ct.c_double),
                ("hx", ct.c_double), ("hy", ct.c_double), ("pad", ct.c_int), ("nzr", ct.c_int),
                ("zr", _dp), ("nu", _dp), ("nzy", ct.c_int), ("zy", _dp), ("kernel_kind", ct.c_int)]


class Sources(ct.Structure):
    _fields_ = [("q", ct.c_int), ("n_points", ct.c_int), ("xyz", _dp), ("A0", ct.c_double)]


class InvertOpts(ct.Structure):
    _fields_ = [("alpha_mode", ct.c_int), ("alpha", ct.c_double), ("alphas", _dp), ("n_alpha", ct.c_int),
                ("delta", ct.c_double), ("tau", ct.c_double), ("output", ct.c_int), ("precision", ct.c_int),
                ("sources", ct.POINTER(Sources)), ("alpha_idx", ct.c_void_p), ("residuals", ct.c_void_p),
                ("info", ct.c_void_p), ("n_bands", ct.c_int), ("net", ct.c_void_p), ("ra", ct.c_int)]


class Instance(ct.Structure):
    _fields_ = [("handle", ct.c_void_p), ("U", ct.c_void_p), ("Q", ct.c_int), ("opts", ct.POINTER(InvertOpts)),
                ("out", ct.c_void_p)]


class Fr3dError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_string(status)} (status {status})")
        self.status = status


_lib = None

# the names the C ABI exports (include/fr3d.h)
EXPORTS = ("fr3d_kernel_transform", "fr3d_handle_destroy", "fr3d_handle_query", "fr3d_fwd_apply",
           "fr3d_fwd_apply_noalloc",
           "fr3d_zeta_from_xi", "fr3d_choose_alpha", "fr3d_invert", "fr3d_invert_host",
           "fr3d_last_launch_count", "fr3d_profile_enable", "fr3d_profile_read", "fr3d_status_string",
           "fr3d_batch_create", "fr3d_batch_run", "fr3d_batch_launch_count", "fr3d_batch_destroy",
           "fr3d_invert_batched", "fr3d_invert_batched_workspace",
           "fr3d_mlp_create", "fr3d_mlp_destroy", "fr3d_mlp_query", "fr3d_mlp_get_params", "fr3d_mlp_set_params",
           "fr3d_mlp_forward", "fr3d_mlp_gradient", "fr3d_mlp_train_step", "fr3d_band_features",
           "fr3d_band_alpha_targets", "fr3d_autotune_mode", "fr3d_autotune_query",
           "fr3d_test_withhold_queue_counts", "fr3d_assemble_rhs",
           "fr3d_unet_create", "fr3d_unet_destroy", "fr3d_unet_query", "fr3d_unet_get_params", "fr3d_unet_set_params",
           "fr3d_unet_forward", "fr3d_unet_gradient", "fr3d_unet_train_step", "fr3d_unet_error_flags")


def load(path: str | None = None):
    """Load libfr3d.so (built by paper_1703_01216_gb300.build); raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build it with paper_1703_01216_gb300.build.build()")
    lib = ct.CDLL(p)
    vp, i, d = ct.c_void_p, ct.c_int, ct.c_double
    lib.fr3d_kernel_transform.argtypes = [ct.POINTER(Geometry), ct.POINTER(vp), vp]
    lib.fr3d_handle_destroy.argtypes = [vp]
    lib.fr3d_handle_destroy.restype = None
    lib.fr3d_handle_query.argtypes = [vp, ct.POINTER(i), ct.POINTER(i), ct.POINTER(i), ct.POINTER(d)]
    lib.fr3d_fwd_apply.argtypes = [vp, vp, i, vp, i, vp]
    lib.fr3d_fwd_apply_noalloc.argtypes = [vp, vp, i, vp, vp]
    lib.fr3d_zeta_from_xi.argtypes = [vp, vp, ct.POINTER(Sources), vp, i, vp]
    lib.fr3d_choose_alpha.argtypes = [vp, vp, i, _dp, i, d, d, i, vp, vp, vp, vp]
    lib.fr3d_invert.argtypes = [vp, vp, i, ct.POINTER(InvertOpts), vp, vp]
    lib.fr3d_invert_host.argtypes = [vp, vp, i, ct.POINTER(InvertOpts), vp, vp]
    lib.fr3d_last_launch_count.argtypes = [vp]
    lib.fr3d_profile_enable.argtypes = [vp, i]
    lib.fr3d_profile_read.argtypes = [vp, ct.POINTER(i), ct.POINTER(ct.c_float), i]
    lib.fr3d_batch_create.argtypes = [ct.POINTER(Instance), i, ct.POINTER(vp), vp]
    lib.fr3d_batch_run.argtypes = [vp, vp]
    lib.fr3d_batch_launch_count.argtypes = [vp]
    lib.fr3d_batch_destroy.argtypes = [vp]
    lib.fr3d_batch_destroy.restype = None
    lib.fr3d_invert_batched.argtypes = [ct.POINTER(Instance), i, vp, ct.c_size_t, vp]
    lib.fr3d_invert_batched_workspace.argtypes = [ct.POINTER(Instance), i, ct.POINTER(ct.c_size_t), vp]
    lib.fr3d_mlp_create.argtypes = [i, i, i, ct.c_ulonglong, ct.POINTER(vp)]
    lib.fr3d_mlp_destroy.argtypes = [vp]
    lib.fr3d_mlp_destroy.restype = None
    lib.fr3d_mlp_query.argtypes = [vp, ct.POINTER(i), ct.POINTER(i), ct.POINTER(i), ct.POINTER(i)]
    lib.fr3d_mlp_get_params.argtypes = [vp, vp]
    lib.fr3d_mlp_set_params.argtypes = [vp, vp]
    lib.fr3d_mlp_forward.argtypes = [vp, vp, i, vp, vp]
    lib.fr3d_mlp_gradient.argtypes = [vp, vp, vp, i, vp, vp, vp]
    lib.fr3d_mlp_train_step.argtypes = [vp, vp, vp, i, ct.c_float, vp, vp]
    lib.fr3d_band_features.argtypes = [vp, vp, i, i, d, vp, vp]
    lib.fr3d_band_alpha_targets.argtypes = [vp, vp, vp, i, _dp, i, i, vp, vp, vp, vp]
    lib.fr3d_autotune_mode.argtypes = [i]
    lib.fr3d_autotune_query.argtypes = [vp, ct.POINTER(i), ct.POINTER(ct.c_float), i]
    lib.fr3d_test_withhold_queue_counts.argtypes = [i]
    lib.fr3d_assemble_rhs.argtypes = [vp, vp, i, ct.POINTER(Sources), d, d, i, d, vp, vp]
    lib.fr3d_unet_create.argtypes = [i, i, i, i, ct.c_float, ct.c_ulonglong, ct.POINTER(vp)]
    lib.fr3d_unet_destroy.argtypes = [vp]
    lib.fr3d_unet_destroy.restype = None
    lib.fr3d_unet_query.argtypes = [vp, ct.POINTER(i)]
    lib.fr3d_unet_get_params.argtypes = [vp, vp]
    lib.fr3d_unet_set_params.argtypes = [vp, vp]
    lib.fr3d_unet_forward.argtypes = [vp, vp, i, vp, vp]
    lib.fr3d_unet_gradient.argtypes = [vp, vp, vp, i, vp, vp, vp]
    lib.fr3d_unet_train_step.argtypes = [vp, vp, vp, i, ct.c_float, vp, vp]
    lib.fr3d_unet_error_flags.argtypes = [vp, ct.POINTER(i)]
    lib.fr3d_status_string.argtypes = [i]
    lib.fr3d_status_string.restype = ct.c_char_p
    for name in EXPORTS:
        if name not in ("fr3d_handle_destroy", "fr3d_status_string", "fr3d_batch_destroy", "fr3d_mlp_destroy",
                        "fr3d_unet_destroy"):
            getattr(lib, name).restype = ct.c_int
    _lib = lib
    return lib


def status_string(status: int) -> str:
    return load().fr3d_status_string(int(status)).decode()


def _check(status: int, what: str):
    if status < 0:
        raise Fr3dError(status, what)
    return status


def _f64(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return a, a.ctypes.data_as(_dp)


def _stream(stream):
    if stream is None:
        import torch
        return ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ct.c_void_p(stream)
    return ct.c_void_p(stream.cuda_stream)


def _need(t, what: str, *, device: bool = True, dtype=None, numel: int | None = None, optional: bool = False):
    """Argument check before a call: a torch tensor (or numpy array for host buffers) must live where the
    C ABI expects it (device or host), be contiguous, have the dtype of the call's precision and hold at
    least the elements the call reads or writes.  A plain integer is a raw address the caller vouches for
    and is passed through unchecked."""
    if t is None:
        if optional:
            return
        raise Fr3dError(-1, f"{what}: missing")
    if isinstance(t, int):
        return
    if isinstance(t, np.ndarray):
        if device:
            raise Fr3dError(-1, f"{what}: a device (CUDA) buffer is required, got a numpy array")
        ok_c, n_el, dt = t.flags["C_CONTIGUOUS"], t.size, t.dtype
        want = None if dtype is None else np.dtype(str(dtype).replace("torch.", ""))
    elif hasattr(t, "data_ptr"):
        if device and not t.is_cuda:
            raise Fr3dError(-1, f"{what}: a device (CUDA) tensor is required, got one on {t.device}")
        if not device and t.is_cuda:
            raise Fr3dError(-1, f"{what}: a host tensor is required, got one on {t.device}")
        ok_c, n_el, dt, want = t.is_contiguous(), t.numel(), t.dtype, dtype
    else:
        raise Fr3dError(-1, f"{what}: unsupported argument type {type(t).__name__}")
    if not ok_c:
        raise Fr3dError(-1, f"{what}: must be contiguous")
    if want is not None and dt != want:
        raise Fr3dError(-1, f"{what}: dtype {dt} does not match the call (expected {want})")
    if numel is not None and n_el < numel:
        raise Fr3dError(-1, f"{what}: {n_el} elements, the call needs {numel}")


def _real_dtype(precision: int):
    import torch
    return torch.float64 if precision == PREC_FP64 else torch.float32


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return ct.c_void_p(t)
    if hasattr(t, "data_ptr"):
        return ct.c_void_p(t.data_ptr())
    if isinstance(t, np.ndarray):
        return ct.c_void_p(t.ctypes.data)
    raise TypeError(type(t))


def make_sources(points, A0: float = 1.0):
    """points [Q, L, 3] -> (Sources, keepalive)."""
    pts, p = _f64(points)
    if pts.ndim != 3 or pts.shape[2] != 3:
        raise ValueError("points must be [Q, L, 3]")
    return Sources(pts.shape[0], pts.shape[1], p, float(A0)), pts


class Handle:
    """Owns an fr3d_handle (fr3d_kernel_transform ... fr3d_handle_destroy)."""

    def __init__(self, n, x0, h, zr, zy, nu=None, stream=None, kind=K_DZ_INV_R, pad=1):
        lib = load()
        self._zr, zrp = _f64(zr)
        self._zy, zyp = _f64(zy)
        if nu is None:
            self._nu, nup = None, None
        else:
            self._nu, nup = _f64(nu)
        g = Geometry(int(n), int(n), float(x0), float(x0), float(h), float(h), int(pad), self._zr.size, zrp, nup,
                     self._zy.size, zyp, int(kind))
        hp = ct.c_void_p()
        _check(lib.fr3d_kernel_transform(ct.byref(g), ct.byref(hp), _stream(stream)), "fr3d_kernel_transform")
        self.ptr = hp
        n_, m_, mp_, s2 = ct.c_int(), ct.c_int(), ct.c_int(), ct.c_double()
        _check(lib.fr3d_handle_query(hp, ct.byref(n_), ct.byref(m_), ct.byref(mp_), ct.byref(s2)), "query")
        self.n, self.M, self.Mp, self.s2 = n_.value, m_.value, mp_.value, s2.value

    def close(self):
        if getattr(self, "ptr", None):
            load().fr3d_handle_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kernel_transform(n, x0, h, zr, zy, nu=None, stream=None, kind=K_DZ_INV_R, pad=1) -> Handle:
    """pad = 1: the periodic box of the n x n grid (Sec. 5); pad = 2: the zero-padded 2n x 2n box."""
    return Handle(n, x0, h, zr, zy, nu, stream, kind, pad)


def fwd_apply(handle: Handle, zeta, Q: int, U, precision: int = PREC_FP32, stream=None):
    n2, dt = handle.n * handle.n, _real_dtype(precision)
    _need(zeta, "zeta", dtype=dt, numel=Q * handle.Mp * n2)
    _need(U, "U", dtype=dt, numel=Q * handle.M * n2)
    _check(load().fr3d_fwd_apply(handle.ptr, _ptr(zeta), int(Q), _ptr(U), int(precision), _stream(stream)),
           "fr3d_fwd_apply")


def fwd_apply_noalloc(handle: Handle, zeta, Q: int, U, stream=None):
    """fr3d_fwd_apply_noalloc: FP32 forward operator using the library's static scratch (no allocation)."""
    import torch
    n2 = handle.n * handle.n
    _need(zeta, "zeta", dtype=torch.float32, numel=Q * handle.Mp * n2)
    _need(U, "U", dtype=torch.float32, numel=Q * handle.M * n2)
    _check(load().fr3d_fwd_apply_noalloc(handle.ptr, _ptr(zeta), int(Q), _ptr(U), _stream(stream)),
           "fr3d_fwd_apply_noalloc")


def zeta_from_xi(handle: Handle, xi, points, zeta, A0: float = 1.0, precision: int = PREC_FP32, stream=None):
    src, keep = make_sources(points, A0)
    n2, dt = handle.n * handle.n, _real_dtype(precision)
    _need(xi, "xi", dtype=dt, numel=handle.Mp * n2)
    _need(zeta, "zeta", dtype=dt, numel=src.q * handle.Mp * n2)
    _check(load().fr3d_zeta_from_xi(handle.ptr, _ptr(xi), ct.byref(src), _ptr(zeta), int(precision),
                                    _stream(stream)), "fr3d_zeta_from_xi")


def choose_alpha(handle: Handle, U, Q: int, alphas, delta: float, tau: float, alpha_idx, residuals=None, info=None,
                 precision: int = PREC_FP32, stream=None):
    import torch
    a, ap = _f64(alphas)
    _need(U, "U", dtype=_real_dtype(precision), numel=Q * handle.M * handle.n * handle.n)
    _need(alpha_idx, "alpha_idx", dtype=torch.int32, numel=1)
    _need(residuals, "residuals", dtype=torch.float64, numel=a.size, optional=True)
    _need(info, "info", dtype=torch.int32, numel=1, optional=True)
    _check(load().fr3d_choose_alpha(handle.ptr, _ptr(U), int(Q), ap, a.size, float(delta), float(tau),
                                    int(precision), _ptr(alpha_idx), _ptr(residuals), _ptr(info), _stream(stream)),
           "fr3d_choose_alpha")


class Opts:
    """Builds fr3d_invert_opts and keeps its host arrays alive."""

    def __init__(self, *, alpha=None, alphas=None, delta=0.0, tau=1.1, output=OUT_XI, precision=PREC_FP32,
                 points=None, A0=1.0, alpha_idx=None, residuals=None, info=None, n_bands=1, given=False, net=None,
                 ra=RA_TIKHONOV):
        o = InvertOpts()
        o.ra = int(ra)
        self._net = net
        if alpha is not None:
            o.alpha_mode, o.alpha = ALPHA_FIXED, float(alpha)
            self._a = None
        else:
            self._a, ap = _f64(alphas)
            o.alpha_mode = ALPHA_LEARNED if net is not None else (ALPHA_GIVEN if given else ALPHA_DISCREPANCY)
            o.alphas, o.n_alpha = ap, self._a.size
            o.net = net.ptr if net is not None else None
        o.n_bands = int(n_bands)
        o.delta, o.tau, o.output, o.precision = float(delta), float(tau), int(output), int(precision)
        if points is not None:
            self._src, self._pts = make_sources(points, A0)
            o.sources = ct.pointer(self._src)
        o.alpha_idx = _ptr(alpha_idx)
        o.residuals = _ptr(residuals)
        o.info = _ptr(info)
        self.c = o
        self._aux = (alpha_idx, residuals, info)

    def check(self, handle: "Handle", Q: int, U, out, device: bool = True):
        """The buffers of one fr3d_invert / fr3d_invert_host call against the handle's sizes."""
        import torch
        o = self.c
        n2, dt = handle.n * handle.n, _real_dtype(o.precision)
        _need(U, "U", device=device, dtype=dt, numel=Q * handle.M * n2)
        _need(out, "out", device=device, dtype=dt, numel=(1 if o.output == OUT_XI else Q) * handle.Mp * n2)
        nb = max(1, o.n_bands)
        na = 1 if o.alpha_mode == ALPHA_FIXED else o.n_alpha
        idx, res, info = self._aux
        _need(idx, "alpha_idx", dtype=torch.int32, numel=nb, optional=o.alpha_mode != ALPHA_GIVEN)
        _need(res, "residuals", dtype=torch.float64, numel=nb * na, optional=True)
        _need(info, "info", dtype=torch.int32, numel=1, optional=True)


def invert(handle: Handle, U, Q: int, out, opts: Opts, stream=None):
    opts.check(handle, Q, U, out)
    _check(load().fr3d_invert(handle.ptr, _ptr(U), int(Q), ct.byref(opts.c), _ptr(out), _stream(stream)),
           "fr3d_invert")


def invert_host(handle: Handle, U_host, Q: int, out_host, opts: Opts, stream=None):
    opts.check(handle, Q, U_host, out_host, device=False)
    _check(load().fr3d_invert_host(handle.ptr, _ptr(U_host), int(Q), ct.byref(opts.c), _ptr(out_host),
                                   _stream(stream)), "fr3d_invert_host")


def last_launch_count(handle: Handle) -> int:
    return int(load().fr3d_last_launch_count(handle.ptr))


STAGE_NAMES = ("row_r2c", "col_fwd", "alpha", "col_solve", "row_c2r", "table", "contract", "col_inv", "other",
               "inv_fused")


def profile_enable(handle: Handle, enable: bool = True):
    _check(load().fr3d_profile_enable(handle.ptr, int(bool(enable))), "fr3d_profile_enable")


def profile_read(handle: Handle, cap: int = 96):
    """[(stage name, ms)] for the launches of the latest call (waits for them)."""
    kinds = (ct.c_int * cap)()
    ms = (ct.c_float * cap)()
    n = _check(load().fr3d_profile_read(handle.ptr, kinds, ms, cap), "fr3d_profile_read")
    return [(STAGE_NAMES[kinds[i]], float(ms[i])) for i in range(n)]


def assemble_rhs(handle: Handle, dV2dz, Q: int, points, A2: float, c0: float, n_pi: int, pi_half: float, U,
                 A0: float = 1.0, stream=None):
    import torch
    src, keep = make_sources(points, A0)
    n = Q * handle.M * handle.n * handle.n
    _need(dV2dz, "dV2dz", dtype=torch.float32, numel=n)
    _need(U, "U", dtype=torch.float32, numel=n)
    _check(load().fr3d_assemble_rhs(handle.ptr, _ptr(dV2dz), int(Q), ct.byref(src), float(A2), float(c0), int(n_pi),
                                    float(pi_half), _ptr(U), _stream(stream)), "fr3d_assemble_rhs")


def autotune_mode(mode: int | None = None) -> int:
    """Set the fused-inverse autotuner mode (0 off, 1 tune per shape, 2 + v force variant v) and return
    the previous one; with no argument, return the current mode."""
    r = load().fr3d_autotune_mode(-1 if mode is None else int(mode))
    _check(r, "fr3d_autotune_mode")
    return r


def autotune_query(handle: Handle):
    """(variant of the handle's last fused inverse, per-variant tuning times in ms or zeros)."""
    v = ct.c_int()
    ms = (ct.c_float * 8)()
    n = load().fr3d_autotune_query(handle.ptr, ct.byref(v), ms, 8)
    _check(n, "fr3d_autotune_query")
    return v.value, [float(ms[k]) for k in range(n)]


def test_withhold_queue_counts(on: bool) -> bool:
    """Test hook of the tile-queue variant's bounded waits (fr3d_test_withhold_queue_counts): while on, its
    row tiles' waits run out and the call reports FR3D_INFO_TIMEOUT.  Returns the previous setting."""
    return bool(load().fr3d_test_withhold_queue_counts(1 if on else 0))


class Mlp:
    """fr3d_mlp: the per-band alpha network (weights on the device)."""

    def __init__(self, n_in: int, n_hidden: int, n_out: int, seed: int = 0):
        p = ct.c_void_p()
        _check(load().fr3d_mlp_create(int(n_in), int(n_hidden), int(n_out), int(seed), ct.byref(p)),
               "fr3d_mlp_create")
        self.ptr = p
        self.n_in, self.n_hidden, self.n_out = int(n_in), int(n_hidden), int(n_out)
        npar = ct.c_int()
        _check(load().fr3d_mlp_query(self.ptr, None, None, None, ct.byref(npar)), "fr3d_mlp_query")
        self.n_params = npar.value

    def get_params(self) -> np.ndarray:
        out = np.empty(self.n_params, np.float32)
        _check(load().fr3d_mlp_get_params(self.ptr, _ptr(out)), "fr3d_mlp_get_params")
        return out

    def set_params(self, params):
        a = np.ascontiguousarray(np.asarray(params, np.float32))
        if a.size != self.n_params:
            raise ValueError("wrong parameter count")
        _check(load().fr3d_mlp_set_params(self.ptr, _ptr(a)), "fr3d_mlp_set_params")

    def forward(self, X, Y, stream=None):
        _check(load().fr3d_mlp_forward(self.ptr, _ptr(X), int(X.shape[0]), _ptr(Y), _stream(stream)),
               "fr3d_mlp_forward")

    def gradient(self, X, T, grad=None, loss=None, stream=None):
        _check(load().fr3d_mlp_gradient(self.ptr, _ptr(X), _ptr(T), int(X.shape[0]), _ptr(grad), _ptr(loss),
                                        _stream(stream)), "fr3d_mlp_gradient")

    def train_step(self, X, T, lr: float, loss=None, stream=None):
        _check(load().fr3d_mlp_train_step(self.ptr, _ptr(X), _ptr(T), int(X.shape[0]), float(lr), _ptr(loss),
                                          _stream(stream)), "fr3d_mlp_train_step")

    def close(self):
        if getattr(self, "ptr", None):
            load().fr3d_mlp_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def band_features(handle: Handle, U, Q: int, n_bands: int, delta: float, feat, stream=None):
    import torch
    _need(U, "U", dtype=torch.float32, numel=Q * handle.M * handle.n * handle.n)
    _need(feat, "feat", dtype=torch.float32, numel=max(1, n_bands))
    _check(load().fr3d_band_features(handle.ptr, _ptr(U), int(Q), int(n_bands), float(delta), _ptr(feat),
                                     _stream(stream)), "fr3d_band_features")


def band_alpha_targets(handle: Handle, U, zeta_true, Q: int, alphas, n_bands: int, idx, target=None, err=None,
                       stream=None):
    import torch
    a, ap = _f64(alphas)
    n2 = handle.n * handle.n
    _need(U, "U", dtype=torch.float32, numel=Q * handle.M * n2)
    _need(zeta_true, "zeta_true", dtype=torch.float32, numel=Q * handle.Mp * n2)
    _need(idx, "idx", dtype=torch.int32, numel=max(1, n_bands))
    _need(target, "target", dtype=torch.float32, numel=max(1, n_bands), optional=True)
    _need(err, "err", dtype=torch.float64, numel=max(1, n_bands) * a.size, optional=True)
    _check(load().fr3d_band_alpha_targets(handle.ptr, _ptr(U), _ptr(zeta_true), int(Q), ap, a.size, int(n_bands),
                                          _ptr(idx), _ptr(target), _ptr(err), _stream(stream)),
           "fr3d_band_alpha_targets")


class Batch:
    """A batch plan over independent instances (fr3d_batch_create ... fr3d_batch_destroy).

    ``items`` is a list of (Handle, U tensor, Q, Opts, out tensor); their device buffers and options
    must stay alive and unchanged while the plan exists."""

    def __init__(self, items, stream=None):
        lib = load()
        self._items = items
        arr = (Instance * len(items))()
        for k, (h, U, Q, opts, out) in enumerate(items):
            arr[k] = Instance(h.ptr.value, U.data_ptr(), int(Q), ct.pointer(opts.c), out.data_ptr())
        self._arr = arr
        bp = ct.c_void_p()
        _check(lib.fr3d_batch_create(arr, len(items), ct.byref(bp), _stream(stream)), "fr3d_batch_create")
        self.ptr = bp

    def run(self, stream=None):
        _check(load().fr3d_batch_run(self.ptr, _stream(stream)), "fr3d_batch_run")

    @property
    def launches(self) -> int:
        return int(load().fr3d_batch_launch_count(self.ptr))

    def close(self):
        if getattr(self, "ptr", None):
            load().fr3d_batch_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Unet:
    """fr3d_unet: the learned post-corrector (weights, optimiser state and activation buffers on the device)."""

    def __init__(self, depth: int, height: int, width: int, max_batch: int, in_scale: float = 1.0, seed: int = 0):
        p = ct.c_void_p()
        _check(load().fr3d_unet_create(int(depth), int(height), int(width), int(max_batch), float(in_scale), int(seed),
                                       ct.byref(p)), "fr3d_unet_create")
        self.ptr = p
        self.shape = (int(depth), int(height), int(width))
        npar = ct.c_int()
        _check(load().fr3d_unet_query(self.ptr, ct.byref(npar)), "fr3d_unet_query")
        self.n_params = npar.value

    def get_params(self) -> np.ndarray:
        out = np.empty(self.n_params, np.float32)
        _check(load().fr3d_unet_get_params(self.ptr, _ptr(out)), "fr3d_unet_get_params")
        return out

    def set_params(self, params):
        a = np.ascontiguousarray(np.asarray(params, np.float32))
        if a.size != self.n_params:
            raise ValueError("wrong parameter count")
        _check(load().fr3d_unet_set_params(self.ptr, _ptr(a)), "fr3d_unet_set_params")

    def _vol(self, t, what, optional=False):
        import torch
        b = int(t.shape[0]) if hasattr(t, "shape") else 1
        _need(t, what, dtype=torch.float32, numel=b * self.shape[0] * self.shape[1] * self.shape[2],
              optional=optional)

    def forward(self, x, y, stream=None):
        self._vol(x, "x")
        self._vol(y, "y")
        _check(load().fr3d_unet_forward(self.ptr, _ptr(x), int(x.shape[0]), _ptr(y), _stream(stream)),
               "fr3d_unet_forward")

    def gradient(self, x, t, grad=None, loss=None, stream=None):
        import torch
        self._vol(x, "x")
        self._vol(t, "t")
        _need(grad, "grad", dtype=torch.float32, numel=self.n_params, optional=True)
        _need(loss, "loss", dtype=torch.float32, numel=1, optional=True)
        _check(load().fr3d_unet_gradient(self.ptr, _ptr(x), _ptr(t), int(x.shape[0]), _ptr(grad), _ptr(loss),
                                         _stream(stream)), "fr3d_unet_gradient")

    def train_step(self, x, t, lr: float, loss=None, stream=None):
        import torch
        self._vol(x, "x")
        self._vol(t, "t")
        _need(loss, "loss", dtype=torch.float32, numel=1, optional=True)
        _check(load().fr3d_unet_train_step(self.ptr, _ptr(x), _ptr(t), int(x.shape[0]), float(lr), _ptr(loss),
                                           _stream(stream)), "fr3d_unet_train_step")

    def error_flags(self) -> int:
        f = ct.c_int()
        _check(load().fr3d_unet_error_flags(self.ptr, ct.byref(f)), "fr3d_unet_error_flags")
        return f.value

    def close(self):
        if getattr(self, "ptr", None):
            load().fr3d_unet_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _instances(items):
    arr = (Instance * len(items))()
    for k, (h, U, Q, opts, out) in enumerate(items):
        arr[k] = Instance(h.ptr.value, U.data_ptr(), int(Q), ct.pointer(opts.c), out.data_ptr())
    return arr


def invert_batched_workspace(items, stream=None) -> int:
    """Bytes of device workspace fr3d_invert_batched needs for these (handle, U, Q, opts, out) items."""
    arr = _instances(items)
    b = ct.c_size_t()
    _check(load().fr3d_invert_batched_workspace(arr, len(items), ct.byref(b), _stream(stream)),
           "fr3d_invert_batched_workspace")
    return int(b.value)


def invert_batched(items, workspace, stream=None):
    """One-shot batched inversion in the caller's device workspace (a uint8 CUDA tensor)."""
    _need(workspace, "workspace")
    arr = _instances(items)
    nbytes = workspace.numel() * workspace.element_size() if hasattr(workspace, "numel") else 0
    _check(load().fr3d_invert_batched(arr, len(items), _ptr(workspace), nbytes, _stream(stream)),
           "fr3d_invert_batched")
