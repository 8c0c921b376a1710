"""FFCz on B300: Python binding of the C-ABI library ``libffcz.so``.

Argument marshalling only: every step of the correction runs in the CUDA
kernels behind the C ABI (``include/ffcz.h``).  PyTorch provides device
memory and the current stream.  There is no CPU fallback: if the library is
missing or no GPU is present, the calls raise.

    import paper_2601_01596_b300 as ffcz
    plan = ffcz.Plan([(512, 512, 512)])
    stats = plan.correct(e, eps_s, eps_f)      # e: float32 CUDA tensor, in place
"""
from __future__ import annotations

import collections.abc
import ctypes
import os
from typing import Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libffcz.so")

OK, ERR_INVALID, ERR_UNSUPPORTED, ERR_CUDA = 0, 1, 2, 3
ERR_NOT_CONVERGED, ERR_CERT_FAILED, ERR_NONFINITE, ERR_TIMEOUT, ERR_OOM = 4, 5, 6, 7, 8

SYMBOLS = ("ffcz_default_opts", "ffcz_plan", "ffcz_set_stream", "ffcz_workspace_bytes",
           "ffcz_correct", "ffcz_correct_host", "ffcz_check", "ffcz_correct_backward",
           "ffcz_destroy", "ffcz_strerror", "ffcz_last_error", "ffcz_launch_count",
           "ffcz_profile_enable", "ffcz_profile_count", "ffcz_profile_entry",
           "ffcz_check_static", "ffcz_plan_describe", "ffcz_edit_layout", "ffcz_edits_dense",
           "ffcz_edits_compact", "ffcz_apply_edits", "ffcz_edits_compact16", "ffcz_apply_edits16",
           "ffcz_correct_pw", "ffcz_power_spectrum_bounds",
           "ffcz_ckpt_floats", "ffcz_correct_ckpt", "ffcz_correct_backward_ckpt", "ffcz_fp64_peak")
STATIC_MAX_POINTS = 1 << 22   # FFCZ_STATIC_MAX_POINTS


class Opts(ctypes.Structure):
    _fields_ = [("max_iters", ctypes.c_int32), ("min_iters", ctypes.c_int32),
                ("shrink", ctypes.c_double), ("precision", ctypes.c_int32),
                ("certify", ctypes.c_int32), ("max_repairs", ctypes.c_int32),
                ("K", ctypes.c_int32), ("ckpt_every", ctypes.c_int32),
                ("chunk", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("count_active", ctypes.c_int32), ("edits", ctypes.c_int32),
                ("pointwise", ctypes.c_int32), ("method", ctypes.c_int32),
                ("keep_masks", ctypes.c_int32)]


# Projection of the loop (ffcz_opts.method): Alg. 1 or one of the
# alternatives Sec. III names.
METHODS = {"pocs": 0, "dykstra": 1, "dr": 2, "douglas_rachford": 2, "admm": 3}


class Stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32),
                ("repairs", ctypes.c_int32), ("certified", ctypes.c_int32),
                ("preclipped", ctypes.c_int32), ("host_copies", ctypes.c_int32),
                ("f_ratio", ctypes.c_double), ("s_ratio", ctypes.c_double),
                ("f_margin64", ctypes.c_double), ("s_margin64", ctypes.c_double),
                ("active_s", ctypes.c_int64), ("active_f", ctypes.c_int64),
                ("ms_total", ctypes.c_float), ("ms_cert", ctypes.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class StatsList(collections.abc.Sequence):
    """Per-item stats of one call: a sequence of dicts built on access (no
    per-item work when the call returns); ``.array`` is the same data as a
    numpy structured array without a copy."""

    def __init__(self, arr):
        self._c = arr

    def __len__(self):
        return len(self._c)

    def __getitem__(self, i):
        if isinstance(i, slice):
            return [self[j] for j in range(*i.indices(len(self)))]
        return self._c[i].as_dict()

    @property
    def array(self):
        import numpy as np
        return np.ctypeslib.as_array(self._c)


_lib = None


def lib() -> ctypes.CDLL:
    """Load ``libffcz.so`` (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run `python -m paper_2601_01596_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
        L.ffcz_default_opts.argtypes = [ctypes.POINTER(Opts)]
        L.ffcz_default_opts.restype = None
        L.ffcz_plan.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(ctypes.c_int64), i64,
                                ctypes.POINTER(Opts), vp]
        L.ffcz_set_stream.argtypes = [vp, vp]
        L.ffcz_workspace_bytes.argtypes = [vp]
        L.ffcz_workspace_bytes.restype = ctypes.c_size_t
        L.ffcz_plan_describe.argtypes = [vp, ctypes.c_char_p, i32]
        L.ffcz_plan_describe.restype = i32
        L.ffcz_edit_layout.argtypes = [vp, i64, ctypes.POINTER(ctypes.c_int64)]
        L.ffcz_edits_dense.argtypes = [vp, vp, vp]
        L.ffcz_edits_compact.argtypes = [vp, i32, vp, vp, vp, vp, ctypes.POINTER(ctypes.c_int64)]
        L.ffcz_apply_edits.argtypes = [vp, vp, dp, dp, i32, vp, vp, vp, vp]
        L.ffcz_edits_compact16.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, ctypes.POINTER(ctypes.c_int64)]
        L.ffcz_apply_edits16.argtypes = [vp, vp, dp, dp, i32, vp, vp, vp, vp, vp, vp,
                                         ctypes.POINTER(ctypes.c_int64)]
        L.ffcz_correct_pw.argtypes = [vp, vp, vp, vp, ctypes.POINTER(Stats)]
        L.ffcz_power_spectrum_bounds.argtypes = [vp, vp, dp, vp]
        L.ffcz_correct.argtypes = [vp, vp, dp, dp, ctypes.POINTER(Stats)]
        L.ffcz_correct_host.argtypes = [vp, vp, dp, dp, ctypes.POINTER(Stats)]
        L.ffcz_check.argtypes = [vp, vp, dp, dp, ctypes.POINTER(Stats)]
        L.ffcz_correct_backward.argtypes = [vp, vp, vp, vp, dp, dp]
        L.ffcz_ckpt_floats.argtypes = [vp]
        L.ffcz_ckpt_floats.restype = ctypes.c_int64
        L.ffcz_correct_ckpt.argtypes = [vp, vp, dp, dp, vp, ctypes.POINTER(Stats)]
        L.ffcz_correct_backward_ckpt.argtypes = [vp, vp, vp, vp, vp, dp, dp]
        L.ffcz_destroy.argtypes = [vp]
        L.ffcz_destroy.restype = None
        L.ffcz_strerror.argtypes = [i32]
        L.ffcz_strerror.restype = ctypes.c_char_p
        L.ffcz_last_error.restype = ctypes.c_char_p
        L.ffcz_launch_count.restype = ctypes.c_int64
        L.ffcz_profile_enable.argtypes = [vp, i32]
        L.ffcz_profile_count.argtypes = [vp]
        L.ffcz_profile_count.restype = ctypes.c_int
        L.ffcz_profile_entry.argtypes = [vp, i32, ctypes.c_char_p, i32,
                                         ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_int64)]
        L.ffcz_check_static.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_int64), ctypes.c_double,
                                        ctypes.c_double, vp, ctypes.POINTER(Stats)]
        L.ffcz_check_static.restype = ctypes.c_int
        L.ffcz_fp64_peak.argtypes = [i32, vp, dp]
        L.ffcz_fp64_peak.restype = ctypes.c_int
        for name in ("ffcz_plan", "ffcz_set_stream", "ffcz_correct", "ffcz_correct_host",
                     "ffcz_check", "ffcz_correct_backward", "ffcz_profile_enable",
                     "ffcz_profile_entry", "ffcz_correct_ckpt", "ffcz_correct_backward_ckpt"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


class FFCzError(RuntimeError):
    def __init__(self, status: int, detail: str = ""):
        self.status = status
        msg = lib().ffcz_strerror(status).decode()
        super().__init__(f"{msg} (status {status}){': ' + detail if detail else ''}")


def _check(status: int, allow=()) -> int:
    if status != OK and status not in allow:
        raise FFCzError(status, lib().ffcz_last_error().decode())
    return status


def default_opts(**kw) -> Opts:
    o = Opts()
    lib().ffcz_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        if k == "method" and isinstance(v, str):
            v = METHODS[v]
        setattr(o, k, v)
    return o


def launch_count() -> int:
    return int(lib().ffcz_launch_count())


def fp64_peak(kind: str = "fma", stream=None) -> float:
    """Measured FP64 rate of the current GPU in flop/s (``ffcz_fp64_peak``):
    ``fma`` (2 flops per instruction) or ``add`` (1)."""
    v = ctypes.c_double()
    _check(lib().ffcz_fp64_peak({"fma": 0, "add": 1}[kind], ctypes.c_void_p(_stream_ptr(stream)),
                                ctypes.byref(v)))
    return float(v.value)


def _dbl(values, n):
    if isinstance(values, (int, float)):
        values = [float(values)] * n
    values = [float(v) for v in values]
    if len(values) != n:
        raise ValueError(f"expected {n} bounds, got {len(values)}")
    return (ctypes.c_double * n)(*values)


def _stream_ptr(stream) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


class Plan:
    """A plan for a batch of fields of one rank (2D or 3D), each axis a power
    of two.  ``shapes``: list of per-item shapes.  Options as in ffcz_opts."""

    def __init__(self, shapes: Sequence[Sequence[int]], stream=None, **opts):
        shapes = [tuple(int(n) for n in s) for s in shapes]
        if not shapes:
            raise ValueError("no items")
        ndim = len(shapes[0])
        if any(len(s) != ndim for s in shapes):
            raise ValueError("all items must have the same rank")
        self.shapes = shapes
        self.ndim = ndim
        self.batch = len(shapes)
        self.sizes = [int(__import__("math").prod(s)) for s in shapes]
        self.total = sum(self.sizes)
        self.opts = default_opts(**opts)
        flat = (ctypes.c_int64 * (self.batch * ndim))(*[n for s in shapes for n in s])
        h = ctypes.c_void_p()
        _check(lib().ffcz_plan(ctypes.byref(h), ndim, flat, self.batch, ctypes.byref(self.opts),
                               ctypes.c_void_p(_stream_ptr(stream))))
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.ffcz_destroy(h)
            self._h = None

    @property
    def workspace_bytes(self) -> int:
        return int(lib().ffcz_workspace_bytes(self._h))

    def edit_layout(self, item: int = -1):
        """(points, bins, s_flag_off, s_code_off, f_flag_off, f_code_off) of one
        item, or the totals / array sizes for item = -1 (plan with edits=1)."""
        out = (ctypes.c_int64 * 6)()
        _check(lib().ffcz_edit_layout(self._h, item, out))
        return tuple(int(x) for x in out)

    def edits_dense(self):
        """Dense edits of the last call: (spatial float32 [points], frequency
        complex64 [half-spectrum bins]) as CUDA tensors."""
        import torch
        tot = self.edit_layout(-1)
        s = torch.empty(tot[0], dtype=torch.float32, device="cuda")
        f = torch.empty(2 * tot[1], dtype=torch.float32, device="cuda")
        _check(lib().ffcz_edits_dense(self._h, ctypes.c_void_p(s.data_ptr()), ctypes.c_void_p(f.data_ptr())))
        return s, torch.view_as_complex(f.view(-1, 2))

    def edits_compact(self, m_bits: int = 16):
        """CompactEdits + QuantizeEdits: dict of CUDA tensors (s_flags, s_codes,
        f_flags, f_codes, regions at ``edit_layout(i)`` offsets) and ``counts``
        (numpy [batch, 2]: nonzero spatial / frequency components per item)."""
        import numpy as np
        import torch
        tot = self.edit_layout(-1)
        d = dict(s_flags=torch.zeros(max(1, tot[2]), dtype=torch.uint8, device="cuda"),
                 s_codes=torch.zeros(max(1, tot[3]), dtype=torch.int32, device="cuda"),
                 f_flags=torch.zeros(max(1, tot[4]), dtype=torch.uint8, device="cuda"),
                 f_codes=torch.zeros(max(1, tot[5]), dtype=torch.int32, device="cuda"))
        counts = (ctypes.c_int64 * (2 * self.batch))()
        _check(lib().ffcz_edits_compact(self._h, m_bits, *[ctypes.c_void_p(d[k].data_ptr()) for k in
                                                         ("s_flags", "s_codes", "f_flags", "f_codes")],
                                        counts))
        d["counts"] = np.array(counts, dtype=np.int64).reshape(self.batch, 2)
        return d

    def edits_compact16(self, m_bits: int = 16):
        """``edits_compact`` with 16-bit codes: dict of CUDA tensors (s_flags,
        s_codes int16, s_wide int32, f_flags, f_codes int16, f_wide int32) and
        ``counts`` (numpy [batch, 4]: nonzero spatial / frequency components,
        spatial / frequency escapes)."""
        import numpy as np
        import torch
        tot = self.edit_layout(-1)
        d = dict(s_flags=torch.zeros(max(1, tot[2]), dtype=torch.uint8, device="cuda"),
                 s_codes=torch.zeros(max(1, tot[3]), dtype=torch.int16, device="cuda"),
                 s_wide=torch.zeros(max(1, tot[3]), dtype=torch.int32, device="cuda"),
                 f_flags=torch.zeros(max(1, tot[4]), dtype=torch.uint8, device="cuda"),
                 f_codes=torch.zeros(max(1, tot[5]), dtype=torch.int16, device="cuda"),
                 f_wide=torch.zeros(max(1, tot[5]), dtype=torch.int32, device="cuda"))
        counts = (ctypes.c_int64 * (4 * self.batch))()
        _check(lib().ffcz_edits_compact16(self._h, m_bits, *[ctypes.c_void_p(d[k].data_ptr()) for k in
                                                           ("s_flags", "s_codes", "s_wide", "f_flags", "f_codes",
                                                            "f_wide")], counts))
        d["counts"] = np.array(counts, dtype=np.int64).reshape(self.batch, 4)
        return d

    def apply_edits16(self, xhat, eps_s, eps_f, stored, m_bits: int = 16, stream=None):
        """``apply_edits`` from ``edits_compact16``'s dict (counts included)."""
        import numpy as np
        self._bind_stream(stream)
        ptrs = [ctypes.c_void_p(stored[k].data_ptr()) for k in ("s_flags", "s_codes", "s_wide", "f_flags",
                                                                "f_codes", "f_wide")]
        c = np.ascontiguousarray(stored["counts"], dtype=np.int64).reshape(-1)
        counts = (ctypes.c_int64 * c.size)(*[int(x) for x in c])
        _check(lib().ffcz_apply_edits16(self._h, self._ptr(xhat, "xhat"), _dbl(eps_s, self.batch),
                                        _dbl(eps_f, self.batch), m_bits, *ptrs, counts))

    def apply_edits(self, xhat, eps_s, eps_f, stored, m_bits: int = 16, stream=None):
        """x_hat += S~ + IFFT(F~) from the stored form (``edits_compact``'s
        dict: s_flags, s_codes, f_flags, f_codes); ``xhat`` float32 CUDA, the
        packed items, updated in place."""
        self._bind_stream(stream)
        ptrs = [ctypes.c_void_p(stored[k].data_ptr()) for k in ("s_flags", "s_codes", "f_flags", "f_codes")]
        _check(lib().ffcz_apply_edits(self._h, self._ptr(xhat, "xhat"), _dbl(eps_s, self.batch),
                                      _dbl(eps_f, self.batch), m_bits, *ptrs))

    def describe(self) -> str:
        """Item groups and the pass variants the tuner chose for them."""
        n = lib().ffcz_plan_describe(self._h, None, 0)
        buf = ctypes.create_string_buffer(n + 1)
        lib().ffcz_plan_describe(self._h, buf, n + 1)
        return buf.value.decode()

    def profile(self, on: bool = True):
        """Turn per-kernel event timing on (clears the table) or off."""
        _check(lib().ffcz_profile_enable(self._h, 1 if on else 0))

    def profile_table(self):
        """{kernel key: (total ms, launches)} accumulated since profile(True)."""
        out = {}
        buf = ctypes.create_string_buffer(64)
        for i in range(lib().ffcz_profile_count(self._h)):
            ms, n = ctypes.c_double(), ctypes.c_int64()
            _check(lib().ffcz_profile_entry(self._h, i, buf, 64, ctypes.byref(ms), ctypes.byref(n)))
            out[buf.value.decode()] = (ms.value, n.value)
        return out

    def _bind_stream(self, stream=None):
        _check(lib().ffcz_set_stream(self._h, ctypes.c_void_p(_stream_ptr(stream))))

    def _ptr(self, t, name):
        import torch
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float32 or not t.is_cuda:
            raise TypeError(f"{name} must be a float32 CUDA tensor")
        if not t.is_contiguous() or t.numel() != self.total:
            raise ValueError(f"{name} must be contiguous with {self.total} elements")
        return ctypes.c_void_p(t.data_ptr())

    def correct(self, e, eps_s, eps_f, stream=None, allow=(ERR_NOT_CONVERGED, ERR_CERT_FAILED,
                                                           ERR_NONFINITE)):
        """Correct ``e`` (packed items, float32 CUDA) in place; per-item stats."""
        self._bind_stream(stream)
        st = (Stats * self.batch)()
        s = lib().ffcz_correct(self._h, self._ptr(e, "e"), _dbl(eps_s, self.batch),
                               _dbl(eps_f, self.batch), st)
        _check(s, allow)
        return StatsList(st)

    def correct_pw(self, e, e_bounds, f_bounds, stream=None, allow=(ERR_NOT_CONVERGED, ERR_CERT_FAILED,
                                                                     ERR_NONFINITE)):
        """Correct ``e`` in place with pointwise bounds (plan made with
        pointwise=1): ``e_bounds`` float32 like ``e``; ``f_bounds`` the
        (Delta^Re, Delta^Im) pairs on every item's half spectrum, complex64 or
        float32 pairs (``edit_layout`` bins, items back to back)."""
        import torch
        self._bind_stream(stream)
        fb = torch.view_as_real(f_bounds) if f_bounds.is_complex() else f_bounds
        nb = self.edit_layout(-1)[1]
        if not (fb.is_cuda and fb.dtype == torch.float32 and fb.is_contiguous() and fb.numel() == 2 * nb):
            raise ValueError(f"f_bounds must be {nb} contiguous complex64 / float32-pair values on the GPU")
        st = (Stats * self.batch)()
        s = lib().ffcz_correct_pw(self._h, self._ptr(e, "e"), self._ptr(e_bounds, "e_bounds"),
                                  ctypes.c_void_p(fb.data_ptr()), st)
        _check(s, allow)
        return StatsList(st)

    def power_spectrum_bounds(self, x, rho, stream=None):
        """Per-bin (Delta^Re, Delta^Im) keeping every power-spectrum shell of
        the original fields ``x`` (float32 CUDA, packed items) within the
        relative bound(s) ``rho``; complex64 CUDA tensor for ``correct_pw``."""
        import torch
        self._bind_stream(stream)
        nb = self.edit_layout(-1)[1]
        out = torch.empty(2 * nb, dtype=torch.float32, device="cuda")
        rho = [rho] * self.batch if isinstance(rho, (int, float)) else rho
        _check(lib().ffcz_power_spectrum_bounds(self._h, self._ptr(x, "x"), _dbl(rho, self.batch),
                                                ctypes.c_void_p(out.data_ptr())))
        return torch.view_as_complex(out.view(-1, 2))

    def correct_host(self, e_np, eps_s, eps_f, allow=(ERR_NOT_CONVERGED, ERR_CERT_FAILED,
                                                      ERR_NONFINITE)):
        """Correct a float32 host array in place through the host-buffer entry point."""
        import numpy as np
        if not isinstance(e_np, np.ndarray) or e_np.dtype != np.float32 or \
                not e_np.flags.c_contiguous or e_np.size != self.total:
            raise TypeError("e_np must be a contiguous float32 array with all items")
        st = (Stats * self.batch)()
        s = lib().ffcz_correct_host(self._h, ctypes.c_void_p(e_np.ctypes.data),
                                    _dbl(eps_s, self.batch), _dbl(eps_f, self.batch), st)
        _check(s, allow)
        return StatsList(st)

    def check(self, e, eps_s, eps_f, stream=None):
        """FP64 certification of ``e``; returns per-item stats (``certified``)."""
        self._bind_stream(stream)
        st = (Stats * self.batch)()
        s = lib().ffcz_check(self._h, self._ptr(e, "e"), _dbl(eps_s, self.batch),
                             _dbl(eps_f, self.batch), st)
        _check(s, (ERR_CERT_FAILED,))
        return StatsList(st)

    def backward(self, e0, grad_out, grad_in, eps_s, eps_f, stream=None, ckpt=None):
        """grad_in <- (d e_K / d e0)^T grad_out for K = opts.K forced iterations
        (``ckpt``: the checkpoints of ``correct_ckpt`` for this e0; else the
        forward runs again to take them)."""
        self._bind_stream(stream)
        if ckpt is None:
            _check(lib().ffcz_correct_backward(self._h, self._ptr(e0, "e0"),
                                               self._ptr(grad_out, "grad_out"),
                                               self._ptr(grad_in, "grad_in"),
                                               _dbl(eps_s, self.batch), _dbl(eps_f, self.batch)))
            return
        self._check_ckpt(ckpt)
        _check(lib().ffcz_correct_backward_ckpt(self._h, self._ptr(e0, "e0"), ctypes.c_void_p(ckpt.data_ptr()),
                                                self._ptr(grad_out, "grad_out"),
                                                self._ptr(grad_in, "grad_in"),
                                                _dbl(eps_s, self.batch), _dbl(eps_f, self.batch)))

    def ckpt_floats(self) -> int:
        """Size (float32 values) of the checkpoint buffer of ``correct_ckpt``."""
        return int(lib().ffcz_ckpt_floats(self._h))

    def _check_ckpt(self, ckpt):
        import torch
        n = self.ckpt_floats()
        if not (isinstance(ckpt, torch.Tensor) and ckpt.is_cuda and ckpt.dtype == torch.float32
                and ckpt.is_contiguous() and ckpt.numel() == n):
            raise ValueError(f"ckpt must be {n} contiguous float32 values on the GPU")

    def correct_ckpt(self, e, eps_s, eps_f, ckpt, stream=None,
                     allow=(ERR_NOT_CONVERGED, ERR_CERT_FAILED, ERR_NONFINITE)):
        """``correct`` for the differentiable form (min_iters = max_iters = K)
        that also writes the backward's checkpoints into ``ckpt``
        (``ckpt_floats()`` float32 values on the GPU)."""
        self._bind_stream(stream)
        self._check_ckpt(ckpt)
        st = (Stats * self.batch)()
        s = lib().ffcz_correct_ckpt(self._h, self._ptr(e, "e"), _dbl(eps_s, self.batch),
                                    _dbl(eps_f, self.batch), ctypes.c_void_p(ckpt.data_ptr()), st)
        _check(s, allow)
        return StatsList(st)


def check_static(e, eps_s: float, eps_f: float, stream=None):
    """FP64 certification of one field without a plan or any device allocation
    (``ffcz_check_static``); returns (status, stats dict)."""
    import torch
    if not isinstance(e, torch.Tensor) or e.dtype != torch.float32 or not e.is_cuda \
            or not e.is_contiguous():
        raise TypeError("e must be a contiguous float32 CUDA tensor")
    shape = (ctypes.c_int64 * e.dim())(*e.shape)
    st = Stats()
    s = lib().ffcz_check_static(ctypes.c_void_p(e.data_ptr()), e.dim(), shape, float(eps_s),
                                float(eps_f), ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(st))
    _check(s, (ERR_CERT_FAILED,))
    return s, st.as_dict()


def correct(e, eps_s, eps_f, **opts):
    """One-shot correction of a single field ``e`` (float32 CUDA tensor) in place."""
    p = Plan([tuple(e.shape)], **opts)
    return p.correct(e.reshape(-1), [eps_s], [eps_f])[0]
