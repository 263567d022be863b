"""ctypes binding of libegt_cpu (include/egt_cpu.h): the FP64 multi-core CPU comparator.

Argument marshalling only; the solver is C++ with OpenMP.  It is a measurement
baseline for the GPU library (bench.py reports it beside the GPU numbers) and is
never called by it.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .egt import STATUS, EGTError, _desc

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libegt_cpu.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "egt_cpu.h")
if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1810_03063_b300.build`")
lib = C.CDLL(LIB_PATH)


class CpuOpts(C.Structure):
    _fields_ = [("alpha", C.c_double), ("eps_mbb", C.c_double), ("max_iters", C.c_int32),
                ("gap_every", C.c_int32), ("threads", C.c_int32)]


class CpuReport(C.Structure):
    _fields_ = [("iters", C.c_int32), ("backoffs", C.c_int32), ("products", C.c_int32), ("threads", C.c_int32),
                ("gap_mbb", C.c_double), ("mu", C.c_double * 2), ("tau", C.c_double), ("seconds", C.c_double)]


_vp = C.c_void_p
lib.egt_cpu_create.argtypes = [_vp, C.POINTER(_vp)]
lib.egt_cpu_destroy.argtypes = [_vp]
lib.egt_cpu_solve.argtypes = [_vp, C.POINTER(CpuOpts), _vp, _vp, C.POINTER(CpuReport)]
lib.egt_cpu_dims.argtypes = [_vp, _vp, _vp]
for _f in (lib.egt_cpu_create, lib.egt_cpu_destroy, lib.egt_cpu_solve, lib.egt_cpu_dims):
    _f.restype = C.c_int
lib.egt_cpu_last_error.argtypes = []
lib.egt_cpu_last_error.restype = C.c_char_p


def _check(st):
    if st != 0:
        raise EGTError(st, lib.egt_cpu_last_error().decode())


class CpuGame:
    """A river endgame compiled for the CPU comparator."""

    def __init__(self, spec):
        d, keep = _desc(spec)
        self._h = _vp()
        _check(lib.egt_cpu_create(C.byref(d), C.byref(self._h)))
        S = (C.c_int32 * 2)()
        H = C.c_int32()
        _check(lib.egt_cpu_dims(self._h, C.cast(S, _vp), C.byref(H)))
        self.S, self.H = (S[0], S[1]), H.value

    def close(self):
        if getattr(self, "_h", None):
            lib.egt_cpu_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, alpha=0.01, eps_mbb=1.0, max_iters=20000, gap_every=1, threads=0, iterates=False):
        """EGT/as from the initial point; returns the report (and x, y [S][H] in input hand
        order with iterates=True)."""
        o = CpuOpts(alpha, eps_mbb, max_iters, gap_every, threads)
        r = CpuReport()
        x = np.empty((self.S[0], self.H)) if iterates else None
        y = np.empty((self.S[1], self.H)) if iterates else None
        st = lib.egt_cpu_solve(self._h, C.byref(o), x.ctypes.data if iterates else None,
                               y.ctypes.data if iterates else None, C.byref(r))
        if st not in (0, 6):
            _check(st)
        out = dict(status=STATUS[st], iters=r.iters, backoffs=r.backoffs, products=r.products, threads=r.threads,
                   gap_mbb=r.gap_mbb, mu=(r.mu[0], r.mu[1]), tau=r.tau, seconds=r.seconds)
        if iterates:
            out.update(x=x, y=y)
        return out
